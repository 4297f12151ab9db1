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
// Two barriers per tile.  Staging: each block is persistent and walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... in row-major order (tiles in flight are spatial neighbours, so
// halo re-reads hit L2).  One thread issues, per tile, two TMA tensor loads into an S-stage ring
// of shared-memory buffers, completion tracked by one mbarrier per stage:
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

#include "gabp_device.cuh"
#include "gabp_internal.h"

namespace gabp {

namespace {

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

// One warp per belief-window row: TY + 2 warps per block.
template <int TY, int S> struct TileLayout {
    static constexpr int TW = TY + 2, TNT = 32 * TW;   // warps, threads
    static constexpr int RX = TTX + 4, RY = TY + 4;   // staged planes (cells), origin (x0-2, y0-2)
    static constexpr int BX = 32, BY = TY + 2;        // belief window, origin (x0-1, y0-1)
    static constexpr int OXW = 40, OY = TY + 3;       // observation index window, origin (xs, y0-2)
    static constexpr uint32_t plane_bytes = 5u * RY * RX * 8u;
    static constexpr uint32_t optr_bytes = (uint32_t)OXW * OY * 4u;
    static constexpr size_t stage = a128(plane_bytes) + a128(optr_bytes);
    // beliefs and observation row ranges are double-buffered (tile parity), so one block-wide
    // barrier per tile separates their writers (phase A) from their readers (phase B)
    static constexpr size_t bel_bytes = sizeof(Belief<float>) * BX * BY;
    static constexpr size_t bel_off = S * stage;
    static constexpr size_t bar_off = a128(bel_off + 2 * bel_bytes);
    static constexpr size_t ints_off = bar_off + 8 * (S + 1);   // S stage barriers + 1 test barrier
    static constexpr int NI = 2 * TY + 2;                         // row starts [TY], prefix [TY + 1], pad
    static constexpr size_t bytes = ints_off + sizeof(int) * (2 * NI + 2);
    static_assert(BY % TW == 0, "window rows must split evenly over the warps");
    static_assert(2 * RX <= 256 && RY <= 256 && OXW <= 256 && OY <= 256, "TMA box dimension above 256");
};

template <int TY, int S>
__global__ void __launch_bounds__(TileLayout<TY, S>::TNT) k_fused_tma(const __grid_constant__ CUtensorMap mplanes,
                                                   const __grid_constant__ CUtensorMap moptr, DevProblem p,
                                                   int src, float beta) {
    using LY = TileLayout<TY, S>;
    constexpr int RX = LY::RX, RY = LY::RY, BX = LY::BX, BY = LY::BY, OXW = LY::OXW;
    constexpr int TW = LY::TW, TNT = LY::TNT;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + LY::bar_off);
    int *flag = reinterpret_cast<int *>(smem + LY::ints_off) + 2 * LY::NI;

    const int nx = p.nx, ny = p.ny;
    const int64_t n = p.n;
    const int ntx = (nx + TTX - 1) / TTX;
    const int ntiles = ntx * ((ny + TY - 1) / TY);
    const int G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *Q = (float2 *)p.P[src ^ 1];
    const float *O = (const float *)p.O[src];
    float *OQ = (float *)p.O[src ^ 1];
    const float var_prior = (float)(1.0 / p.gamma);
    const float aC_in = (float)p.aC[4];

    auto issue = [&](int stage, int tile) {
        const int x0 = (tile % ntx) * TTX, y0 = (tile / ntx) * TY;
        unsigned char *base = smem + stage * LY::stage;
        const uint32_t bar = smem_addr(&bars[stage]);
        mbar_expect_tx(bar, LY::plane_bytes + LY::optr_bytes);
        tma_load_3d(smem_addr(base), &mplanes, 2 * (x0 - 2), y0 - 2, 0, bar);
        tma_load_2d(smem_addr(base + a128(LY::plane_bytes)), &moptr, (x0 - 2) & ~3, y0 - 2, bar);
    };

    if (tid == 0) {
        for (int s = 0; s <= S; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        *flag = 0;
    }
    __syncthreads();
    if (p.debug_stall) {
        // failure-detection test: wait on a barrier that nothing arrives on, before any copy is
        // issued; the bounded wait runs out, the block raises the error flag and returns
        if (tid == 0 && !mbar_wait(smem_addr(&bars[S]), 0, 1LL << 22)) {
            *flag = 1;
            atomicExch(p.err, 1);
        }
        __syncthreads();
        if (*flag) return;
    }
    if (tid == 0)
        for (int s = 0; s < S; ++s) {
            const int t = blockIdx.x + s * G;
            if (t < ntiles) issue(s, t);
        }

    int it = 0;
    bool failed = false;
    for (;; ++it) {
        const int tile = blockIdx.x + it * G;
        if (tile >= ntiles) break;
        const int stage = it % S;
        // a thread whose wait ran out skips phase A (its staged indices may be stale) and the
        // barrier after phase A stops the whole block
        const bool ok = mbar_wait(smem_addr(&bars[stage]), (uint32_t)((it / S) & 1));
        Belief<float> *sb = reinterpret_cast<Belief<float> *>(smem + LY::bel_off + (it & 1) * LY::bel_bytes);
        int *rstart = reinterpret_cast<int *>(smem + LY::ints_off) + (it & 1) * LY::NI;   // [TY]
        int *rpre = rstart + TY;                                                          // [TY + 1]

        const int x0 = (tile % ntx) * TTX, y0 = (tile / ntx) * TY;
        const int xs = (x0 - 2) & ~3;
        const float2 *sm = reinterpret_cast<const float2 *>(smem + stage * LY::stage);   // [5][RY][RX]
        const int *W = reinterpret_cast<const int *>(smem + stage * LY::stage + a128(LY::plane_bytes));
        auto wptr = [&](int x, int y) { return W[(y - y0 + 2) * OXW + (x - xs)]; };

        // ---- A: observation ranges of the tile's rows (last warp), beliefs of the window ----
        if (ok && p.m > 0 && warp == TW - 1) {
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
            Belief<float> b;
            if (ok && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                const int rx = lane + 1, ry = ly + 1;
                float2 m = sm[(DIR_C * RY + ry) * RX + rx];
                CompSum<float> se(m.x), sl(m.y);
                // zero-filled outside the grid: the boundary terms add exact zeros
                m = sm[(DIR_E * RY + ry) * RX + rx - 1]; se.add(m.x); sl.add(m.y);
                m = sm[(DIR_W * RY + ry) * RX + rx + 1]; se.add(m.x); sl.add(m.y);
                m = sm[(DIR_N * RY + ry - 1) * RX + rx]; se.add(m.x); sl.add(m.y);
                m = sm[(DIR_S * RY + ry + 1) * RX + rx]; se.add(m.x); sl.add(m.y);
                if (p.m > 0) {
                    const bool last = gx == nx - 1;
                    const int a0 = wptr(gx, gy);
                    add_obs_pair(se, sl, O, gx > 0 ? wptr(gx - 1, gy) : a0, a0, last ? a0 : wptr(gx + 1, gy), 1, 0);
                    if (gy > 0) {
                        const int c0 = wptr(gx, gy - 1);
                        add_obs_pair(se, sl, O, gx > 0 ? wptr(gx - 1, gy - 1) : c0, c0, last ? c0 : wptr(gx + 1, gy - 1), 3, 2);
                    }
                }
                se.finish();
                sl.finish();
                b.ehi = se.hi; b.elo = se.lo; b.lhi = sl.hi; b.llo = sl.lo;
            } else {
                b.ehi = b.elo = b.lhi = b.llo = 0.f;
            }
            sb[ly * BX + lane] = b;
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        // every thread has finished tile it-1: refill its stage with tile it-1+S
        if (tid == 0 && it > 0) {
            const int t2 = blockIdx.x + (it - 1 + S) * G;
            if (t2 < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue((it - 1) % S, t2);
            }
        }

        // ---- B: cell factors of the tile, then the observation factors based in it ----
        for (int ty = warp; ty < TY; ty += TW) {
            const int tx = lane, gx = x0 + tx, gy = y0 + ty;
            if (tx >= TTX || gx >= nx || gy >= ny) continue;
            const int64_t c = (int64_t)gy * nx + gx;
            const Belief<float> *bs[5] = {&sb[(ty + 1) * BX + tx + 1], &sb[(ty + 1) * BX + tx],
                                          &sb[(ty + 1) * BX + tx + 2], &sb[ty * BX + tx + 1],
                                          &sb[(ty + 2) * BX + tx + 1]};
            float2 own[5];
#pragma unroll
            for (int u = 0; u < 5; ++u) own[u] = sm[(u * RY + ty + 2) * RX + tx + 2];
            const bool inner = gx > 0 && gx < nx - 1 && gy > 0 && gy < ny - 1;
            float a[5];
            if (inner) {
                a[0] = aC_in; a[1] = -1.f; a[2] = -1.f; a[3] = -1.f; a[4] = -1.f;
            } else {
                a[0] = (float)p.aC[grid_degree(gy, gx, nx, ny)];
                a[1] = gx > 0 ? -1.f : 0.f;
                a[2] = gx < nx - 1 ? -1.f : 0.f;
                a[3] = gy > 0 ? -1.f : 0.f;
                a[4] = gy < ny - 1 ? -1.f : 0.f;
            }
            float lam[5], eta[5];
#pragma unroll
            for (int u = 0; u < 5; ++u) {
                if (a[u] != 0.f) {
                    cavity(*bs[u], own[u].x, own[u].y, eta[u], lam[u]);
                } else {
                    lam[u] = 1.f;
                    eta[u] = 0.f;
                }
            }
            float L[5], E[5];
            factor_messages<float, 5>(a, var_prior, 0.f, lam, eta, L, E);
#pragma unroll
            for (int u = 0; u < 5; ++u) {
                float2 out;
                if (a[u] != 0.f) {
                    out.x = damp(own[u].x, E[u], beta);
                    out.y = damp(own[u].y, L[u], beta);
                } else {
                    out.x = 0.f;
                    out.y = 0.f;
                }
                __stcs(Q + u * n + c, out);
            }
        }
        if (p.m > 0) {
            const int total = rpre[TY];
            const float *Wt = (const float *)p.ow;
            const float *YV = (const float *)p.ovar;
            // observation factors go first to the warps without a cell row
            for (int q = (tid + TNT - 32 * TY) % TNT; q < total; q += TNT) {
                int lo = 0, hi = TY - 1;   // last row r with rpre[r] <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (rpre[mid] <= q) lo = mid;
                    else hi = mid - 1;
                }
                const int r = lo;
                const int64_t k = rstart[r] + (q - rpre[r]);
                const int bx = p.obase[k] - (y0 + r) * nx;
                const int lx = bx - x0 + 1, ly = r + 1;   // window coordinates of the base node
                const Belief<float> *ob[4] = {&sb[ly * BX + lx], &sb[ly * BX + lx + 1], &sb[(ly + 1) * BX + lx],
                                              &sb[(ly + 1) * BX + lx + 1]};
                const float4 w4 = *reinterpret_cast<const float4 *>(Wt + 4 * k);
                const float aw[4] = {w4.x, w4.y, w4.z, w4.w};
                const float4 oe4 = *reinterpret_cast<const float4 *>(O + 8 * k);
                const float4 ol4 = *reinterpret_cast<const float4 *>(O + 8 * k + 4);
                const float oe[4] = {oe4.x, oe4.y, oe4.z, oe4.w};
                const float ol[4] = {ol4.x, ol4.y, ol4.z, ol4.w};
                float olam[4], oeta[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) cavity(*ob[u], oe[u], ol[u], oeta[u], olam[u]);
                float OL[4], OE[4];
                const float2 yv = *reinterpret_cast<const float2 *>(YV + 2 * k);
                factor_messages<float, 4>(aw, yv.y, yv.x, olam, oeta, OL, OE);
                float4 ne, nl;
                ne.x = damp(oe[0], OE[0], beta); ne.y = damp(oe[1], OE[1], beta);
                ne.z = damp(oe[2], OE[2], beta); ne.w = damp(oe[3], OE[3], beta);
                nl.x = damp(ol[0], OL[0], beta); nl.y = damp(ol[1], OL[1], beta);
                nl.z = damp(ol[2], OL[2], beta); nl.w = damp(ol[3], OL[3], beta);
                *reinterpret_cast<float4 *>(OQ + 8 * k) = ne;
                *reinterpret_cast<float4 *>(OQ + 8 * k + 4) = nl;
            }
        }
    }

    if (failed && tid == 0) {
        atomicExch(p.err, 1);
        // drain this block's outstanding copies (bounded): the prologue issued tiles 0 .. S-1 and
        // the barrier of tile i >= 1 tile i-1+S, so tiles it .. jmax may be in flight
        const int jmax = it == 0 ? S - 1 : it + S - 2;
        for (int j = it; j <= jmax; ++j) {
            const int t = blockIdx.x + j * G;
            if (t >= ntiles) break;
            mbar_wait(smem_addr(&bars[j % S]), (uint32_t)((j / S) & 1));
        }
    }
}

template <int TY, int S>
cudaError_t launch_cfg(const DevProblem &p, const TmaMaps &maps, int src, double beta, cudaStream_t st) {
    using LY = TileLayout<TY, S>;
    static int grid_cache = 0;
    static int configured_dev = -1;
    // the tensor maps' boxes must have been encoded for this tile height (the smem layout and
    // the expected transaction bytes depend on it)
    if (maps.tx != TTX || maps.ty != TY) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(k_fused_tma<TY, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::bytes);
        if (e != cudaSuccess) return e;
        int nsm = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_tma<TY, S>, LY::TNT, LY::bytes);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cache = nsm * per_sm;
        configured_dev = dev;
    }
    const int ntiles = ((p.nx + TTX - 1) / TTX) * ((p.ny + TY - 1) / TY);
    const int grid = ntiles < grid_cache ? ntiles : grid_cache;
    k_fused_tma<TY, S><<<grid, LY::TNT, LY::bytes, st>>>(maps.planes[src], maps.optr, p, src, (float)beta);
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

// Tensor maps of both message buffers (3-D: 2 nx floats x ny rows x 5 planes) and of the
// observation index (2-D: nx x ny int32 of optr[0..n)), with boxes for the tile shape.
cudaError_t make_tma_maps(const DevProblem &p, int tx, int ty, TmaMaps &maps) {
    maps.valid = false;
    if (!tma_shape_supported(tx, ty)) return cudaErrorInvalidValue;
    auto enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    for (int b = 0; b < 2; ++b) {
        cuuint64_t dims[3] = {(cuuint64_t)2 * p.nx, (cuuint64_t)p.ny, 5};
        cuuint64_t strides[2] = {(cuuint64_t)p.nx * 8, (cuuint64_t)p.n * 8};
        cuuint32_t box[3] = {(cuuint32_t)(2 * (tx + 4)), (cuuint32_t)(ty + 4), 5};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&maps.planes[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p.P[b], dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    cuuint64_t dims[2] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny};
    cuuint64_t strides[1] = {(cuuint64_t)p.nx * 4};
    cuuint32_t box[2] = {40, (cuuint32_t)(ty + 3)};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&maps.optr, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, (void *)p.optr, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    maps.tx = tx;
    maps.ty = ty;
    maps.valid = true;
    return cudaSuccess;
}

size_t tma_smem_bytes(int tx, int ty) {
    if (tx != TTX) return 0;
    if (ty == 14) return TileLayout<14, 2>::bytes;
    if (ty == 22) return TileLayout<22, 2>::bytes;
    if (ty == 30) return TileLayout<30, 2>::bytes;
    return 0;
}

cudaError_t launch_tma_iteration(const DevProblem &p, const TmaMaps &maps, int src, double beta,
                                 cudaStream_t st) {
    if (!maps.valid) return cudaErrorInvalidValue;
    if (maps.ty == 14) return launch_cfg<14, 2>(p, maps, src, beta, st);
    if (maps.ty == 22) return launch_cfg<22, 2>(p, maps, src, beta, st);
    if (maps.ty == 30) return launch_cfg<30, 2>(p, maps, src, beta, st);
    return cudaErrorInvalidValue;
}

}  // namespace gabp
