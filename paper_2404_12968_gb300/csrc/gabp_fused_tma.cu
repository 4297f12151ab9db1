// Fused GaBP iteration, FP32, persistent blocks fed by TMA, warp-per-row tiles.
//
// Work unit: a tile of 30 columns x TY rows of cells.  The nodes its factors touch form a
// 32 x (TY+2) window (the tile plus a one-cell halo), so one warp covers one window row with
// every lane busy.  Per tile the block
//   A. computes the compensated beliefs of the window: one warp per window row (TY + 2 warps),
//      lane = column; prior messages come from the staged planes, observation messages from
//      global memory through the staged observation index;
//   B. updates the tile's cell factors (warp w takes tile row w, lanes 0..29) and
//      the observation factors based in the tile (one per thread), writing the damped messages
//      to the other ping-pong buffer.
// One block barrier per tile (beliefs are double-buffered).  Schedule: the tile rows are cut
// into bands of `run` rows; a run is one tile column of one band, and the runs are dealt to
// the persistent blocks round-robin in band-major order, so that all blocks sweep the grid
// together (tiles in flight are spatial neighbours and halo re-reads hit L2) and every block
// walks down its run tile by tile.  Inside a run the two top rows of a tile's belief window are
// the two bottom rows of the previous tile's window: they are copied, not recomputed.  One
// thread issues, per tile, two TMA tensor loads into an S-stage ring of shared-memory buffers,
// completion tracked by one mbarrier per stage:
//   * the 5 message planes over the tile plus a 2-cell halo, one 3-D box of
//     2 x 34 floats x (TY+4) rows x 5 planes, zero-filled outside the grid;
//   * the observation index (observations before each base cell) over a 40 x (TY+3) box whose
//     x origin is rounded down to a multiple of 4 (16-byte aligned start).
// The zero fill makes the boundary terms of the belief sums exact zeros (adding an exact zero
// leaves a TwoSum unchanged), so the sums need no boundary tests and match the other kernels
// bit for bit.  Every mbarrier wait is bounded; on timeout the kernel raises the error flag,
// waits (bounded) for its own outstanding copies and returns.
//
// Requirements (checked on the host): FP32 messages, nx a multiple of 4.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "gabp_device.cuh"
#include "gabp_internal.h"
#include "gabp_packed.cuh"

namespace gabp {

namespace {

using namespace tiles;

constexpr int TTX = 30;   // tile width in cells: window width 32

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait on phase `parity` of an mbarrier: gives up after `limit` clock cycles
// (default 2^32, about two seconds).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = 1LL << 32) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__host__ __device__ constexpr size_t a128(size_t x) { return (x + 127) & ~size_t(127); }


// Update of the rank-1 factor of one cell (row of L, Eq. 5 / App. A): cavities of its five
// slots from the compensated beliefs, the factor-to-variable messages, damping, and a
// streaming store of the five outgoing messages (planes pn apart).  Slots with a = 0 (missing
// neighbours at the grid border) send (0, 0).
__device__ __forceinline__ void cell_factor(const float (&a)[5], const Belief2 *const (&bs)[5], const float2 (&own)[5],
                                            float var, float r, float2 beta2, float2 *q, int64_t pn) {
    float2 cav[5];
#pragma unroll
    for (int u = 0; u < 5; ++u) cav[u] = a[u] != 0.f ? cavity2(*bs[u], own[u]) : f2(0.f, 1.f);
    float2 msg[5];
    factor_messages2<5, true>(a, var, r, cav, msg);
#pragma unroll
    for (int u = 0; u < 5; ++u) __stcs(q + u * pn, a[u] != 0.f ? damp2(own[u], msg[u], beta2) : f2(0.f, 0.f));
}

// The same update reading the cell's own messages from the staged planes (plane u at
// own[u * ostride]) where they are needed instead of holding them in registers across the
// factor update (the batched kernel: 2 % faster there, 1 % slower for one problem).
__device__ __forceinline__ void cell_factor_sm(const float (&a)[5], const Belief2 *const (&bs)[5], const float2 *own,
                                               int ostride, float var, float r, float2 beta2, float2 *q, int64_t pn) {
    float2 cav[5];
#pragma unroll
    for (int u = 0; u < 5; ++u) cav[u] = a[u] != 0.f ? cavity2(*bs[u], own[u * ostride]) : f2(0.f, 1.f);
    float2 msg[5];
    factor_messages2<5, true>(a, var, r, cav, msg);
#pragma unroll
    for (int u = 0; u < 5; ++u)
        __stcs(q + u * pn, a[u] != 0.f ? damp2(own[u * ostride], msg[u], beta2) : f2(0.f, 0.f));
}

// RW belief-window rows (and up to RW cell rows) per warp: (TY + 2) / RW warps per block.
template <int TY, int S, int RW> struct TileLayout {
    static constexpr int TW = (TY + 2) / RW, TNT = 32 * TW;   // warps, threads
    static constexpr int RX = TTX + 4, RY = TY + 4;   // staged planes (cells), origin (x0-2, y0-2)
    static constexpr int BX = 32, BY = TY + 2;        // belief window, origin (x0-1, y0-1)
    static constexpr int OXW = 40, OY = TY + 3;       // observation index window, origin (xs, y0-2)
    static constexpr uint32_t plane_bytes = 5u * RY * RX * 8u;
    static constexpr uint32_t optr_bytes = (uint32_t)OXW * OY * 4u;
    static constexpr size_t stage = a128(plane_bytes) + a128(optr_bytes);
    // beliefs and observation row ranges are double-buffered (tile parity), so one block-wide
    // barrier per tile separates their writers (phase A) from their readers (phase B)
    static constexpr size_t bel_bytes = sizeof(Belief2) * BX * BY;
    static constexpr size_t bel_off = S * stage;
    static constexpr size_t bar_off = a128(bel_off + 2 * bel_bytes);
    static constexpr size_t ints_off = bar_off + 8 * (S + 1);   // S stage barriers + 1 test barrier
    static constexpr int NI = 2 * TY + 2;                         // row starts [TY], prefix [TY + 1], pad
    static constexpr size_t bytes = ints_off + sizeof(int) * (2 * NI + 2);
    // resident blocks per SM that threads and shared memory (228 KB, 1 KB reserved per block)
    // allow; the register budget is sized for it
    static constexpr int MINB_T = 2048 / TNT, MINB_S = (int)((228 * 1024) / (bytes + 1024));
    static constexpr int MINB = MINB_T < MINB_S ? MINB_T : MINB_S;
    static_assert(BY == RW * TW, "window rows must split evenly over the warps");
    static_assert(2 * RX <= 256 && RY <= 256 && OXW <= 256 && OY <= 256, "TMA box dimension above 256");
};

// BATCH: the tiles of several problems (TmaBatchArgs) instead of one; the per-tile work is the
// same, on the problem that owns the tile.
template <int TY, int S, int RW, bool BATCH>
__global__ void __launch_bounds__(TileLayout<TY, S, RW>::TNT, TileLayout<TY, S, RW>::MINB)
    k_fused_tma(const __grid_constant__ CUtensorMap mplanes, const __grid_constant__ CUtensorMap moptr,
                const __grid_constant__ DevProblem p, const __grid_constant__ TmaBatchArgs ba, const TileRuns tr,
                int src, float beta) {
    using LY = TileLayout<TY, S, RW>;
    constexpr int RX = LY::RX, RY = LY::RY, BX = LY::BX, BY = LY::BY, OXW = LY::OXW;
    constexpr int TW = LY::TW, TNT = LY::TNT;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + LY::bar_off);
    int *flag = reinterpret_cast<int *>(smem + LY::ints_off) + 2 * LY::NI;

    const int ntiles = BATCH ? *ba.nitems : 0;   // BATCH: work items
    const int G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2 beta2 = f2(beta, beta);

    // BATCH: work item -> (problem, tile column, tile row, carry flag)
    auto locate = [&](int item) { return ba.items[item]; };

    // single problem (thread 0): the two tensor loads of tile (cx, cy)
    auto issue = [&](int stage, int cx, int cy) {
        unsigned char *base = smem + stage * LY::stage;
        const uint32_t bar = smem_addr(&bars[stage]);
        const int x0 = cx * TTX, y0 = cy * TY;
        mbar_expect_tx(bar, LY::plane_bytes + LY::optr_bytes);
        tma_load_3d(smem_addr(base), &mplanes, 2 * (x0 - 2), y0 - 2, 0, bar);
        tma_load_2d(smem_addr(base + a128(LY::plane_bytes)), &moptr, (x0 - 2) & ~3, y0 - 2, bar);
    };

    // BATCH (thread 0): the message planes and the observation index of the tile's problem by
    // the tensor copies of its own maps (every member's plane rows are padded to an even pitch,
    // its index rows to a multiple of 4 ints, so both have 16-byte row strides)
    auto fill = [&](int stage, int item) {
        if (tid != 0) return;
        unsigned char *base = smem + stage * LY::stage;
        const uint32_t bar = smem_addr(&bars[stage]);
        const int4 w = locate(item);
        const int prob = w.x;
        const int x0 = w.y * TTX, y0 = w.z * TY;
        mbar_expect_tx(bar, LY::plane_bytes + LY::optr_bytes);
        tma_load_3d(smem_addr(base), &ba.maps[prob].planes[src], 2 * (x0 - 2), y0 - 2, 0, bar);
        tma_load_2d(smem_addr(base + a128(LY::plane_bytes)), &ba.maps[prob].optr, (x0 - 2) & ~3, y0 - 2, bar);
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(smem_addr(&bars[s]), 1);
        mbar_init(smem_addr(&bars[S]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        *flag = 0;
    }
    __syncthreads();
    if (BATCH ? ba.debug_stall : p.debug_stall) {
        // failure-detection test: wait on a barrier that nothing arrives on, before any copy is
        // issued; the bounded wait runs out, the block raises the error flag and returns
        if (tid == 0 && !mbar_wait(smem_addr(&bars[S]), 0, 1LL << 22)) {
            *flag = 1;
            atomicExch(BATCH ? ba.err : p.err, 1);
        }
        __syncthreads();
        if (*flag) return;
    }
    TileWalk wk{0, 0, 0, 0};   // single problem: this block's tile
    if constexpr (BATCH) {
        for (int s = 0; s < S; ++s) {
            const int t = blockIdx.x + s * G;
            if (t >= ntiles) break;
            fill(s, t);
        }
    } else {
        wk.start(blockIdx.x, tr);
        if (tid == 0) {
            TileWalk w = wk;
            for (int s = 0; s < S && w.len > 0; ++s, w.next(tr)) issue(s, w.cx, w.ty(tr));
        }
    }

    int it = 0;
    bool failed = false;
    for (;; ++it) {
        // the tile's problem: the kernel parameter, or (BATCH) the table entry of its problem
        int4 w = make_int4(0, 0, 0, 0);   // BATCH: the work item
        if constexpr (BATCH) {
            const int tile = blockIdx.x + it * G;
            if (tile >= ntiles) break;
            w = locate(tile);
        } else {
            if (it > 0) wk.next(tr);
            if (wk.len == 0) break;
        }
        // inside a run: window rows 0 and 1 are rows TY and TY + 1 of the previous tile's window
        const bool carry = BATCH ? w.w != 0 : wk.r > 0;
        const DevProblem &cur = BATCH ? ba.table[w.x] : p;
        const int nx = cur.nx, ny = cur.ny;
        const int64_t pn = cur.pn, m = cur.m;
        float2 *const Q = (float2 *)cur.P[src ^ 1];
        const float *const O = (const float *)cur.O[src];
        float *const OQ = (float *)cur.O[src ^ 1];
        const float var_prior = cur.var_f;
        const float aC_in = cur.aC_f[4];
        const int stage = it % S;
        // a thread whose wait ran out skips phase A (its staged indices may be stale) and the
        // barrier after phase A stops the whole block
        const bool ok = mbar_wait(smem_addr(&bars[stage]), (uint32_t)((it / S) & 1));
        Belief2 *sb = reinterpret_cast<Belief2 *>(smem + LY::bel_off + (it & 1) * LY::bel_bytes);
        const Belief2 *sbp = reinterpret_cast<const Belief2 *>(smem + LY::bel_off + ((it & 1) ^ 1) * LY::bel_bytes);
        int *rstart = reinterpret_cast<int *>(smem + LY::ints_off) + (it & 1) * LY::NI;   // [TY]
        int *rpre = rstart + TY;                                                          // [TY + 1]

        const int x0 = (BATCH ? w.y : wk.cx) * TTX;
        const int y0 = (BATCH ? w.z : wk.ty(tr)) * TY;
        const int xs = (x0 - 2) & ~3;
        const float2 *sm = reinterpret_cast<const float2 *>(smem + stage * LY::stage);   // [5][RY][RX]
        const int *W = reinterpret_cast<const int *>(smem + stage * LY::stage + a128(LY::plane_bytes));
        auto wptr = [&](int x, int y) { return W[(y - y0 + 2) * OXW + (x - xs)]; };

        // ---- A: observation ranges of the tile's rows (last warp, or the first when it only
        // copies its row), beliefs of the window ----
        if (ok && m > 0 && warp == (carry ? 0 : TW - 1)) {
            int st = 0, cnt = 0;
            const int gy = y0 + lane;
            if (lane < TY && gy < ny) {
                st = wptr(x0, gy);
                cnt = wptr(min(x0 + TTX, nx - 1), gy) - st;
                if (cnt < 0) cnt = 0;
            }
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            if (lane < TY) {
                rstart[lane] = st;
                rpre[lane] = inc - cnt;
            }
            if (lane == TY - 1) rpre[TY] = inc;
        }
        for (int ly = warp; ly < BY; ly += TW) {
            const int gx = x0 - 1 + lane, gy = y0 - 1 + ly;
            Belief2 b;
            if (carry && ly < 2) {
                b = sbp[(ly + TY) * BX + lane];
            } else if (ok && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                const int rx = lane + 1, ry = ly + 1;
                // observation ranges of the node: base row gy (corners 1, 0) and base row gy-1
                // (corners 3, 2; row -1 of the staged index is zero-filled, an empty range).  The
                // first two messages of each range are loaded before the prior sums, so that their
                // latency overlaps them (the order of the sum is unchanged).  A missing candidate
                // is (-0, -0): adding -0 leaves a TwoSum's value unchanged, so the first candidates
                // are added without a branch; the second ones only when some lane of the warp has
                // one (a warp vote), as most warps have none.
                int lo1 = 0, mid1 = 0, hi1 = 0, lo2 = 0, mid2 = 0, hi2 = 0;
                const float2 nz = f2(-0.f, -0.f);
                float2 first1 = nz, first2 = nz, second1 = nz, second2 = nz;
                bool any2 = false;
                if (m > 0) {
                    const bool last = gx == nx - 1;
                    mid1 = wptr(gx, gy);
                    lo1 = gx > 0 ? wptr(gx - 1, gy) : mid1;
                    hi1 = last ? mid1 : wptr(gx + 1, gy);
                    mid2 = wptr(gx, gy - 1);
                    lo2 = gx > 0 ? wptr(gx - 1, gy - 1) : mid2;
                    hi2 = last ? mid2 : wptr(gx + 1, gy - 1);
                    const float2 *O2 = reinterpret_cast<const float2 *>(O);   // (eta, Lambda) of k, corner c at 4 k + c
                    if (lo1 < hi1) first1 = O2[4 * (int64_t)lo1 + (lo1 < mid1 ? 1 : 0)];
                    if (lo2 < hi2) first2 = O2[4 * (int64_t)lo2 + (lo2 < mid2 ? 3 : 2)];
                    any2 = __any_sync(__activemask(), lo1 + 1 < hi1 || lo2 + 1 < hi2);
                    if (any2) {
                        if (lo1 + 1 < hi1) second1 = O2[4 * (int64_t)(lo1 + 1) + (lo1 + 1 < mid1 ? 1 : 0)];
                        if (lo2 + 1 < hi2) second2 = O2[4 * (int64_t)(lo2 + 1) + (lo2 + 1 < mid2 ? 3 : 2)];
                    }
                }
                CompSum2 s(sm[(DIR_C * RY + ry) * RX + rx]);
                // zero-filled outside the grid: the boundary terms add exact zeros
                s.add(sm[(DIR_E * RY + ry) * RX + rx - 1]);
                s.add(sm[(DIR_W * RY + ry) * RX + rx + 1]);
                s.add(sm[(DIR_N * RY + ry - 1) * RX + rx]);
                s.add(sm[(DIR_S * RY + ry + 1) * RX + rx]);
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
                b.hi = s.hi;
                b.lo = s.lo;
            } else {
                b.hi = b.lo = f2(0.f, 0.f);
            }
            sb[ly * BX + lane] = b;
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        // every thread has finished tile it-1: refill its stage with tile it-1+S
        if (it > 0) {
            if constexpr (BATCH) {
                const int t2 = blockIdx.x + (it - 1 + S) * G;
                if (t2 < ntiles) {
                    if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    fill((it - 1) % S, t2);
                }
            } else if (tid == 0) {
                TileWalk w = wk;
                for (int j = 1; j < S; ++j) w.next(tr);
                if (w.len > 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue((it - 1) % S, w.cx, w.ty(tr));
                }
            }
        }

        // ---- B: cell factors of the tile, then the observation factors based in it ----
        for (int ty = warp; ty < TY; ty += TW) {
            const int tx = lane, gx = x0 + tx, gy = y0 + ty;
            if (tx >= TTX || gx >= nx || gy >= ny) continue;
            const int64_t c = (int64_t)gy * nx + gx, pc = (int64_t)gy * cur.px + gx;
            const Belief2 *bs[5] = {&sb[(ty + 1) * BX + tx + 1], &sb[(ty + 1) * BX + tx],
                                          &sb[(ty + 1) * BX + tx + 2], &sb[ty * BX + tx + 1],
                                          &sb[(ty + 2) * BX + tx + 1]};
            if constexpr (BATCH) {
                const float tg = cur.ptgt ? ((const float *)cur.ptgt)[c] : 0.f;   // the cell factor's target
                const float2 *os = sm + (ty + 2) * RX + tx + 2;   // own messages: plane u at os[u * RY * RX]
                if (gx > 0 && gx < nx - 1 && gy > 0 && gy < ny - 1) {
                    const float a[5] = {aC_in, -1.f, -1.f, -1.f, -1.f};
                    cell_factor_sm(a, bs, os, RY * RX, var_prior, tg, beta2, Q + pc, pn);
                } else {
                    const float a[5] = {cur.aC_f[grid_degree(gy, gx, nx, ny)], gx > 0 ? -1.f : 0.f,
                                        gx < nx - 1 ? -1.f : 0.f, gy > 0 ? -1.f : 0.f, gy < ny - 1 ? -1.f : 0.f};
                    cell_factor_sm(a, bs, os, RY * RX, var_prior, tg, beta2, Q + pc, pn);
                }
            } else {
                float2 own[5];
#pragma unroll
                for (int u = 0; u < 5; ++u) own[u] = sm[(u * RY + ty + 2) * RX + tx + 2];
                const float tg = cur.ptgt ? ((const float *)cur.ptgt)[c] : 0.f;   // the cell factor's target
                if (gx > 0 && gx < nx - 1 && gy > 0 && gy < ny - 1) {
                    // interior cell: literal coefficients, so the compiler folds the -1 factors
                    const float a[5] = {aC_in, -1.f, -1.f, -1.f, -1.f};
                    cell_factor(a, bs, own, var_prior, tg, beta2, Q + pc, pn);
                } else {
                    const float a[5] = {cur.aC_f[grid_degree(gy, gx, nx, ny)], gx > 0 ? -1.f : 0.f,
                                        gx < nx - 1 ? -1.f : 0.f, gy > 0 ? -1.f : 0.f, gy < ny - 1 ? -1.f : 0.f};
                    cell_factor(a, bs, own, var_prior, tg, beta2, Q + pc, pn);
                }
            }
        }
        if (m > 0) {
            const int total = rpre[TY];
            const float *Wt = (const float *)cur.ow;
            const float *YV = (const float *)cur.ovar;
            const int *ob = cur.obase;
            // observation factors go first to the two warps with one cell row fewer
            for (int q = (tid + TNT - 32 * (TW - 2)) % TNT; q < total; q += TNT) {
                int lo = 0, hi = TY - 1;   // last row r with rpre[r] <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (rpre[mid] <= q) lo = mid;
                    else hi = mid - 1;
                }
                const int r = lo;
                const int64_t k = rstart[r] + (q - rpre[r]);
                const int bx = ob[k] - (y0 + r) * nx;
                const int lx = bx - x0 + 1, ly = r + 1;   // window coordinates of the base node
                const Belief2 *ob[4] = {&sb[ly * BX + lx], &sb[ly * BX + lx + 1], &sb[(ly + 1) * BX + lx],
                                              &sb[(ly + 1) * BX + lx + 1]};
                obs_factor2(ob, Wt, YV, O, OQ, k, beta2);
            }
        }
    }

    if (failed && tid == 0) {
        atomicExch(BATCH ? ba.err : p.err, 1);
        // drain this block's outstanding copies (bounded): the prologue issued tiles 0 .. S-1 and
        // the barrier of tile i >= 1 tile i-1+S, so tiles it .. jmax may be in flight
        const int jmax = it == 0 ? S - 1 : it + S - 2;
        TileWalk w = wk;
        for (int j = it; j <= jmax; ++j) {
            if constexpr (BATCH) {
                if (blockIdx.x + j * G >= ntiles) break;
            } else {
                if (w.len == 0) break;
                w.next(tr);
            }
            mbar_wait(smem_addr(&bars[j % S]), (uint32_t)((j / S) & 1));
        }
    }
}

// persistent grid of k_fused_tma<TY, S, RW, BATCH>: SMs x resident blocks (set up once per device)
template <int TY, int S, int RW, bool BATCH> cudaError_t persistent_grid(int &grid) {
    using LY = TileLayout<TY, S, RW>;
    static int grid_cache = 0;
    static int configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(k_fused_tma<TY, S, RW, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)LY::bytes);
        if (e != cudaSuccess) return e;
        int nsm = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_tma<TY, S, RW, BATCH>, LY::TNT, LY::bytes);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cache = nsm * per_sm;
        configured_dev = dev;
    }
    grid = grid_cache;
    return cudaSuccess;
}

template <int TY, int S, int RW>
cudaError_t launch_cfg(const DevProblem &p, const TmaMaps &maps, int src, double beta, cudaStream_t st) {
    using LY = TileLayout<TY, S, RW>;
    // the tensor maps' boxes must have been encoded for this tile height (the smem layout and
    // the expected transaction bytes depend on it)
    if (maps.tx != TTX || maps.ty != TY) return cudaErrorInvalidValue;
    if (maps.run < 1) return cudaErrorInvalidValue;
    int grid = 0;
    cudaError_t e = persistent_grid<TY, S, RW, false>(grid);
    if (e != cudaSuccess) return e;
    TileRuns tr;
    tr.run = maps.run;
    tr.ntx = (p.nx + TTX - 1) / TTX;
    tr.nty = (p.ny + TY - 1) / TY;
    const int64_t runs = (int64_t)tr.ntx * ((tr.nty + tr.run - 1) / tr.run);
    if (runs < grid) grid = (int)runs;
    tr.step_x = grid % tr.ntx;
    tr.step_b = grid / tr.ntx;
    const TmaBatchArgs none{};
    k_fused_tma<TY, S, RW, false><<<grid, LY::TNT, LY::bytes, st>>>(maps.planes[src], maps.optr, p, none, tr, src,
                                                                     (float)beta);
    return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

bool tma_shape_supported(int tx, int ty) { return tx == TTX && (ty == 14 || ty == 22 || ty == 30); }

bool tma_problem_supported(const DevProblem &p) { return p.prec == 0 && p.nx % 4 == 0 && p.nx >= 4; }

// Tensor maps of both message buffers (3-D: 2 nx floats x ny rows x 5 planes, rows px cells
// apart) and of the observation index (2-D: nx x ny int32 of optr[0..n)), with boxes for the
// tile shape.
cudaError_t make_tma_maps(const DevProblem &p, int tx, int ty, TmaMaps &maps, int parts, const int *optr,
                          int optr_pitch) {
    maps.valid = false;
    if (!tma_shape_supported(tx, ty)) return cudaErrorInvalidValue;
    auto enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    for (int b = 0; b < 2 && (parts & TMA_MAP_PLANES); ++b) {
        cuuint64_t dims[3] = {(cuuint64_t)2 * p.nx, (cuuint64_t)p.ny, 5};
        cuuint64_t strides[2] = {(cuuint64_t)p.px * 8, (cuuint64_t)p.pn * 8};
        cuuint32_t box[3] = {(cuuint32_t)(2 * (tx + 4)), (cuuint32_t)(ty + 4), 5};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&maps.planes[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p.P[b], dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    if (parts & TMA_MAP_OPTR) {
        cuuint64_t dims[2] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny};
        cuuint64_t strides[1] = {(cuuint64_t)(optr ? optr_pitch : p.nx) * 4};
        cuuint32_t box[2] = {40, (cuuint32_t)(ty + 3)};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&maps.optr, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, (void *)(optr ? optr : p.optr), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    maps.tx = tx;
    maps.ty = ty;
    maps.run = 1;
    maps.valid = true;
    return cudaSuccess;
}

namespace {
// Run length of the single-problem schedule on grid x ty-row tiles: among 1..4 the one whose
// busiest block has the fewest tiles (ties: the longer run, which recomputes fewer belief rows).
template <int TY> int choose_run(int nx, int ny) {
    int grid = 0;
    if (persistent_grid<TY, 2, 1, false>(grid) != cudaSuccess || grid < 1) return 1;
    const int ntx = (nx + TTX - 1) / TTX, nty = (ny + TY - 1) / TY;
    int best = 1;
    int64_t best_load = INT64_MAX;
    std::vector<int64_t> load;
    for (int run = 1; run <= 4; ++run) {
        const int64_t nb = (nty + run - 1) / run, runs = (int64_t)ntx * nb;
        const int64_t g = runs < grid ? runs : grid;
        load.assign((size_t)g, 0);
        for (int64_t u = 0; u < runs; ++u) load[(size_t)(u % g)] += std::min<int64_t>(run, nty - (u / ntx) * run);
        const int64_t worst = *std::max_element(load.begin(), load.end());
        if (worst <= best_load) {
            best_load = worst;
            best = run;
        }
    }
    return best;
}
}  // namespace

int tma_choose_run(const DevProblem &p, int ty) {
    if (ty == 14) return choose_run<14>(p.nx, p.ny);
    if (ty == 22) return choose_run<22>(p.nx, p.ny);
    if (ty == 30) return choose_run<30>(p.nx, p.ny);
    return 1;
}

template <int TY>
cudaError_t launch_batch_cfg(const TmaBatchArgs &ba, const DevProblem &first, int max_tiles, int src, double beta,
                             cudaStream_t st) {
    using LY = TileLayout<TY, 2, 1>;
    int grid = 0;
    cudaError_t e = persistent_grid<TY, 2, 1, true>(grid);
    if (e != cudaSuccess) return e;
    if (max_tiles < grid) grid = max_tiles;
    CUtensorMap unused;
    std::memset(&unused, 0, sizeof unused);
    const TileRuns none{1, 1, 1, 0, 0};
    k_fused_tma<TY, 2, 1, true><<<grid, LY::TNT, LY::bytes, st>>>(unused, unused, first, ba, none, src, (float)beta);
    return cudaGetLastError();
}

bool tma_batch_shape_supported(int ty) { return ty == 14 || ty == 22 || ty == 30; }

int tma_batch_grid(int ty, int max_tiles) {
    int grid = 0;
    if (ty == 14 && persistent_grid<14, 2, 1, true>(grid) != cudaSuccess) return 0;
    if (ty == 22 && persistent_grid<22, 2, 1, true>(grid) != cudaSuccess) return 0;
    if (ty == 30 && persistent_grid<30, 2, 1, true>(grid) != cudaSuccess) return 0;
    if (!tma_batch_shape_supported(ty)) return 0;
    return max_tiles < grid ? max_tiles : grid;
}

// Batched iteration over the 30 x ty tiles of the active problems.  `first` is any one problem
// of the batch (it stands in for the kernel's single-problem parameters, of which batch mode
// reads only nx); max_tiles bounds *nitems (the tiles of all problems).
cudaError_t launch_tma_batch(const TmaBatchArgs &ba, const DevProblem &first, int ty, int max_tiles, int src,
                             double beta, cudaStream_t st) {
    if (max_tiles <= 0) return cudaSuccess;
    if (!ba.maps || !ba.table || !ba.items || !ba.nitems || !ba.err || first.nx < 1) return cudaErrorInvalidValue;
    if (ty == 14) return launch_batch_cfg<14>(ba, first, max_tiles, src, beta, st);
    if (ty == 22) return launch_batch_cfg<22>(ba, first, max_tiles, src, beta, st);
    if (ty == 30) return launch_batch_cfg<30>(ba, first, max_tiles, src, beta, st);
    return cudaErrorInvalidValue;
}

size_t tma_smem_bytes(int tx, int ty) {
    if (tx != TTX) return 0;
    if (ty == 14) return TileLayout<14, 2, 1>::bytes;
    if (ty == 22) return TileLayout<22, 2, 1>::bytes;
    if (ty == 30) return TileLayout<30, 2, 1>::bytes;
    return 0;
}

cudaError_t launch_tma_iteration(const DevProblem &p, const TmaMaps &maps, int src, double beta,
                                 cudaStream_t st) {
    if (!maps.valid) return cudaErrorInvalidValue;
    if (maps.ty == 14) return launch_cfg<14, 2, 1>(p, maps, src, beta, st);
    if (maps.ty == 22) return launch_cfg<22, 2, 1>(p, maps, src, beta, st);
    if (maps.ty == 30) return launch_cfg<30, 2, 1>(p, maps, src, beta, st);
    return cudaErrorInvalidValue;
}

}  // namespace gabp
