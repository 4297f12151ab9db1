// Fused GaBP iteration for the alpha = 4 prior (cell factors = rows of L^2 over 13 slots,
// Sec. 3.1 with alpha / 2 = 2), FP32, persistent blocks walking down tile columns.
//
// Work unit: a tile of 28 columns x TY rows of cells.  The nodes its factors touch (a cell
// factor reaches two steps away; an observation factor based in the tile reaches one step right
// and one down) form a 32 x (TY + 4) window, the tile plus a two-cell halo, so one warp covers
// one window row with every lane busy.  Per tile the block
//   A. computes the compensated beliefs of the window: one warp per window row, lane = column;
//      node v adds slot d of the factor of cell v - offset(d) for d = 0..12 (the 13 incoming
//      prior messages, in slot order), then its observation messages in increasing observation
//      index (corners 1, 0 from base row y, then 3, 2 from base row y - 1);
//   B. updates the tile's cell factors (28 x 8 tiles: cell t on thread t, 7 full warps; 28 x 4:
//      warp w takes tile row w, lanes 0..27) and then the observation factors based in the
//      tile, writing the damped messages to the other buffer.
// Beliefs (and the tile rows' observation ranges) are double-buffered by tile parity, so one
// block barrier per tile separates their writers from their readers.  Inside a run (consecutive
// tiles of one tile column) window rows 0..3 of a tile are rows TY..TY+3 of the previous tile's
// window: they are copied, not recomputed.  The runs are dealt to the persistent blocks
// round-robin in band-major order (tiles in flight are spatial neighbours, so the halo re-reads
// of the message planes hit L2).
//
// The message planes are read through the caches, not staged: the 13 planes of a window with its
// own two-cell halo would take most of an SM's shared memory per block.  Phase A reads plane d
// of every window node's source cell; phase B re-reads the tile cells' own messages, which phase A
// has just brought into L1.
//
// Arithmetic: every belief and message goes through the roundings of the split kernels
// (k_beliefs_l2, k_prior_l2 and k_obs in gabp_split.cu), so the messages are bit-identical to
// theirs.  No kernel here waits on anything but its own block barrier.
//
// Requirements (checked on the host): FP32 messages, planes unpadded (px = nx).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "gabp_device.cuh"
#include "gabp_internal.h"
#include "gabp_l2.cuh"
#include "gabp_packed.cuh"

namespace gabp {

namespace {

using namespace tiles;

constexpr int LTX = 28;   // tile width in cells: window width 32

// Update of the 13-slot cell factor of cell (i, j) (row c of L^2, Sec. 3.1 / App. A), the
// arithmetic of k_prior_l2 with the beliefs read from the window (bc = the cell's own node; slot
// d's node at bc[dy * 32 + dx]): the 13 own messages (own[d * pn]) are loaded together, then
// the cavities, factor_messages with var = 1 / gamma and target 0, damping, and streaming stores
// of the outgoing messages (q[d * pn]).  (Scalar, as the split kernel: the packed two-lane form
// of these formulas measured 30 % slower here, with more registers live across the slot loops.)
// INTERIOR: the cell is two or more cells from the border.
template <bool INTERIOR>
__device__ __forceinline__ void cell_factor_l2(const DevProblem &p, int i, int j, const Belief2 *bc, const float2 *own,
                                               float2 *q, int64_t pn, float var, float beta) {
    float a[L2_SLOTS], lam[L2_SLOTS], eta[L2_SLOTS];
    float2 ow[L2_SLOTS];
#pragma unroll
    for (int d = 0; d < L2_SLOTS; ++d) {
        a[d] = l2_coef_t<float, INTERIOR>(p, i, j, d);
        ow[d] = own[d * pn];
    }
#pragma unroll
    for (int d = 0; d < L2_SLOTS; ++d) {
        if (INTERIOR || a[d] != 0.f) {
            const Belief2 b2 = bc[l2_dy(d) * 32 + l2_dx(d)];
            Belief<float> b;
            b.ehi = b2.hi.x;
            b.lhi = b2.hi.y;
            b.elo = b2.lo.x;
            b.llo = b2.lo.y;
            cavity(b, ow[d].x, ow[d].y, eta[d], lam[d]);
        } else {
            lam[d] = 1.f;
            eta[d] = 0.f;
        }
    }
    float L[L2_SLOTS], E[L2_SLOTS];
    factor_messages<float, L2_SLOTS>(a, var, 0.f, lam, eta, L, E);
#pragma unroll
    for (int d = 0; d < L2_SLOTS; ++d) {
        float2 out = f2(0.f, 0.f);
        if (INTERIOR || a[d] != 0.f) out = f2(damp(ow[d].x, E[d], beta), damp(ow[d].y, L[d], beta));
        __stcs(q + d * pn, out);
    }
}

// Compensated belief of node v = (gy, gx): the 13 incoming prior messages in slot order (slot d
// of the factor of cell v - offset(d), where that cell exists), then its observation messages.
// INTERIOR: every source cell exists (the node is two or more cells from the border).
template <bool INTERIOR>
__device__ __forceinline__ Belief2 node_belief_l2(const float2 *P, const float *O, const int *optr, int64_t pn,
                                                   int64_t m, int nx, int ny, int gx, int gy) {
    const int64_t v = (int64_t)gy * nx + gx;
    // observation ranges of the node: base row gy (corners 1, 0) and base row gy - 1 (corners
    // 3, 2); their first messages are loaded before the prior sums so that the latency overlaps
    // them.  A missing candidate is (-0, -0), which leaves a TwoSum's value unchanged; the second
    // candidates are loaded and added only when some lane of the warp has one.
    int lo1 = 0, mid1 = 0, hi1 = 0, lo2 = 0, mid2 = 0, hi2 = 0;
    const float2 nz = f2(-0.f, -0.f);
    float2 first1 = nz, first2 = nz, second1 = nz, second2 = nz;
    bool any2 = false;
    if (m > 0) {
        mid1 = optr[v];
        lo1 = gx > 0 ? optr[v - 1] : mid1;
        hi1 = optr[v + 1];   // base cells never have x = nx - 1: at the row's end this is mid1
        if (gy > 0) {
            mid2 = optr[v - nx];
            lo2 = gx > 0 ? optr[v - nx - 1] : mid2;
            hi2 = optr[v - nx + 1];
        }
        const float2 *O2 = reinterpret_cast<const float2 *>(O);   // (eta, Lambda) of k, corner c at 4 k + c
        if (lo1 < hi1) first1 = O2[4 * (int64_t)lo1 + (lo1 < mid1 ? 1 : 0)];
        if (lo2 < hi2) first2 = O2[4 * (int64_t)lo2 + (lo2 < mid2 ? 3 : 2)];
        any2 = __any_sync(__activemask(), lo1 + 1 < hi1 || lo2 + 1 < hi2);
        if (any2) {
            if (lo1 + 1 < hi1) second1 = O2[4 * (int64_t)(lo1 + 1) + (lo1 + 1 < mid1 ? 1 : 0)];
            if (lo2 + 1 < hi2) second2 = O2[4 * (int64_t)(lo2 + 1) + (lo2 + 1 < mid2 ? 3 : 2)];
        }
    }
    float2 in[L2_SLOTS];
#pragma unroll
    for (int d = 0; d < L2_SLOTS; ++d) {
        const int ci = gy - l2_dy(d), cj = gx - l2_dx(d);
        in[d] = f2(0.f, 0.f);
        if (INTERIOR || (ci >= 0 && ci < ny && cj >= 0 && cj < nx))
            in[d] = P[d * pn + v - ((int64_t)l2_dy(d) * nx + l2_dx(d))];
    }
    CompSum2 s(in[0]);
#pragma unroll
    for (int d = 1; d < L2_SLOTS; ++d) {
        const int ci = gy - l2_dy(d), cj = gx - l2_dx(d);
        if (INTERIOR || (ci >= 0 && ci < ny && cj >= 0 && cj < nx)) s.add(in[d]);
    }
    if (m > 0) {
        s.add(first1);
        if (any2) {
            s.add(second1);
            if (lo1 + 2 < hi1) add_obs_pair2(s, O, lo1 + 2, mid1, hi1, 1, 0);
        }
        s.add(first2);
        if (any2) {
            s.add(second2);
            if (lo2 + 2 < hi2) add_obs_pair2(s, O, lo2 + 2, mid2, hi2, 3, 2);
        }
    }
    s.finish();
    Belief2 b;
    b.hi = s.hi;
    b.lo = s.lo;
    return b;
}

// Blocks of 32 TY threads (one warp per tile row), registers bounded for 24 resident warps per SM.
template <int TY>
__global__ void __launch_bounds__(32 * TY, 24 / TY)
    k_fused_l2(const __grid_constant__ DevProblem p, const TileRuns tr, int src, float beta) {
    constexpr int BX = 32, BY = TY + 4, TW = TY, TNT = 32 * TY;
    __shared__ Belief2 sbel[2][BY * BX];
    __shared__ int sints[2][2 * TY + 2];   // per parity: row starts [TY], prefix [TY + 1]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = p.nx, ny = p.ny;
    const int64_t pn = p.pn, m = p.m;
    const float2 *const P = (const float2 *)p.P[src];
    float2 *const Q = (float2 *)p.P[src ^ 1];
    const float *const O = (const float *)p.O[src];
    float *const OQ = (float *)p.O[src ^ 1];
    const int *const optr = p.optr;
    const float2 beta2 = f2(beta, beta);
    const float var = p.var_f;

    TileWalk wk;
    wk.start(blockIdx.x, tr);
    for (int it = 0; wk.len > 0; ++it, wk.next(tr)) {
        const bool carry = wk.r > 0;
        const int x0 = wk.cx * LTX, y0 = wk.ty(tr) * TY;
        Belief2 *sb = sbel[it & 1];
        const Belief2 *sbp = sbel[(it & 1) ^ 1];
        int *rstart = sints[it & 1];
        int *rpre = rstart + TY;

        // ---- A: observation ranges of the tile's rows (last warp), beliefs of the window ----
        if (m > 0 && warp == TW - 1) {
            int st = 0, cnt = 0;
            const int gy = y0 + lane;
            if (lane < TY && gy < ny) {
                const int64_t rb = (int64_t)gy * nx;
                st = optr[rb + x0];
                cnt = optr[rb + min(x0 + LTX, nx)] - st;
            }
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            if (lane < TY) {
                rstart[lane] = st;
                rpre[lane] = inc - cnt;
            }
            if (lane == TY - 1) rpre[TY] = inc;
        }
        if (carry)
            for (int ly = warp; ly < 4; ly += TW) sb[ly * BX + lane] = sbp[(ly + TY) * BX + lane];
        // every window node's 13 source cells lie in the grid
        const bool interior = x0 >= 4 && x0 + 32 <= nx && y0 >= 4 && y0 + TY + 4 <= ny;
        for (int ly = (carry ? 4 : 0) + warp; ly < BY; ly += TW) {
            const int gx = x0 - 2 + lane, gy = y0 - 2 + ly;
            Belief2 b;
            if (interior) {
                b = node_belief_l2<true>(P, O, optr, pn, m, nx, ny, gx, gy);
            } else if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                if (gx >= 2 && gx < nx - 2 && gy >= 2 && gy < ny - 2) b = node_belief_l2<true>(P, O, optr, pn, m, nx, ny, gx, gy);
                else b = node_belief_l2<false>(P, O, optr, pn, m, nx, ny, gx, gy);
            } else {
                b.hi = b.lo = f2(0.f, 0.f);
            }
            sb[ly * BX + lane] = b;
        }
        __syncthreads();

        // ---- B: cell factors of the tile, then the observation factors based in it.  When the
        // tile's cells fill whole warps (28 x 8: 224 cells, 7 warps), cell t of the tile runs on
        // thread t and the remaining warp starts the observation factors; otherwise warp w takes
        // tile row w on lanes 0..27 ----
        constexpr int NC = LTX * TY;
        constexpr bool LINEAR = NC % 32 == 0 && NC < TNT;
        auto cell = [&](int tx, int ty) {
            const int gx = x0 + tx, gy = y0 + ty;
            if (gx < nx && gy < ny) {
                const int64_t c = (int64_t)gy * nx + gx;
                const Belief2 *bc = &sb[(ty + 2) * BX + tx + 2];
                if (gx >= 2 && gx < nx - 2 && gy >= 2 && gy < ny - 2)
                    cell_factor_l2<true>(p, gy, gx, bc, P + c, Q + c, pn, var, beta);
                else
                    cell_factor_l2<false>(p, gy, gx, bc, P + c, Q + c, pn, var, beta);
            }
        };
        if constexpr (LINEAR) {
            if (tid < NC) cell(tid % LTX, tid / LTX);
        } else {
            if (lane < LTX) cell(lane, warp);
        }
        if (m > 0) {
            const int total = rpre[TY];
            for (int q = LINEAR ? (tid + TNT - NC) % TNT : tid; q < total; q += TNT) {
                int lo = 0, hi = TY - 1;   // last row r with rpre[r] <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (rpre[mid] <= q) lo = mid;
                    else hi = mid - 1;
                }
                const int r = lo;
                const int64_t k = rstart[r] + (q - rpre[r]);
                const int bx = (int)(p.obase[k] - (int64_t)(y0 + r) * nx);
                const int lx = bx - x0 + 2, ly = r + 2;   // window coordinates of the base node
                const Belief2 *bn[4] = {&sb[ly * BX + lx], &sb[ly * BX + lx + 1], &sb[(ly + 1) * BX + lx],
                                        &sb[(ly + 1) * BX + lx + 1]};
                obs_factor2(bn, (const float *)p.ow, (const float *)p.ovar, O, OQ, k, beta2);
            }
        }
    }
}

// persistent grid of k_fused_l2<TY>: SMs x resident blocks (set up once per device)
template <int TY> cudaError_t l2_persistent_grid(int &grid) {
    static int grid_cache = 0;
    static int configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        // shared memory is only the belief windows: leave the rest of the SM's storage to L1,
        // which holds the message planes between phase A and phase B
        e = cudaFuncSetAttribute(k_fused_l2<TY>, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
        if (e != cudaSuccess) return e;
        int nsm = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_l2<TY>, 32 * TY, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cache = nsm * per_sm;
        configured_dev = dev;
    }
    grid = grid_cache;
    return cudaSuccess;
}

// Run length for nx x ny on 28 x TY tiles: among 1, 2, 4, 8 and 16 the one whose busiest block
// has the least phase-A work (TY + 4 window rows for a run's first tile, TY for the others).
template <int TY> int l2_choose_run(int nx, int ny, int grid) {
    const int ntx = (nx + LTX - 1) / LTX, nty = (ny + TY - 1) / TY;
    int best = 1;
    int64_t best_load = INT64_MAX;
    std::vector<int64_t> load;
    for (int run : {1, 2, 4, 8, 16}) {
        const int64_t nb = (nty + run - 1) / run, runs = (int64_t)ntx * nb;
        const int64_t g = runs < grid ? runs : grid;
        load.assign((size_t)g, 0);
        for (int64_t u = 0; u < runs; ++u) {
            const int64_t len = std::min<int64_t>(run, nty - (u / ntx) * run);
            load[(size_t)(u % g)] += len * TY + 4;
        }
        const int64_t worst = *std::max_element(load.begin(), load.end());
        if (worst <= best_load) {
            best_load = worst;
            best = run;
        }
    }
    return best;
}

template <int TY> cudaError_t launch_l2_cfg(const DevProblem &p, int run, int src, double beta, cudaStream_t st) {
    int grid = 0;
    cudaError_t e = l2_persistent_grid<TY>(grid);
    if (e != cudaSuccess) return e;
    TileRuns tr;
    tr.ntx = (p.nx + LTX - 1) / LTX;
    tr.nty = (p.ny + TY - 1) / TY;
    tr.run = run;
    const int64_t runs = (int64_t)tr.ntx * ((tr.nty + tr.run - 1) / tr.run);
    if (runs < grid) grid = (int)runs;
    tr.step_x = grid % tr.ntx;
    tr.step_b = grid / tr.ntx;
    k_fused_l2<TY><<<grid, 32 * TY, 0, st>>>(p, tr, src, (float)beta);
    return cudaGetLastError();
}

}  // namespace

bool fused_l2_shape_supported(int ty) { return ty == 4 || ty == 8; }

int fused_l2_choose_run(const DevProblem &p, int ty) {
    int grid = 0;
    if (ty == 8 && l2_persistent_grid<8>(grid) == cudaSuccess) return l2_choose_run<8>(p.nx, p.ny, grid);
    if (ty == 4 && l2_persistent_grid<4>(grid) == cudaSuccess) return l2_choose_run<4>(p.nx, p.ny, grid);
    return 1;
}

cudaError_t launch_fused_l2_iteration(const DevProblem &p, int ty, int run, int src, double beta, cudaStream_t st) {
    if (p.order != 2 || p.prec != 0 || p.px != p.nx || p.nx < 1 || p.ny < 1 || run < 1) return cudaErrorInvalidValue;
    if (ty == 8) return launch_l2_cfg<8>(p, run, src, beta, st);
    if (ty == 4) return launch_l2_cfg<4>(p, run, src, beta, st);
    return cudaErrorInvalidValue;
}

}  // namespace gabp
