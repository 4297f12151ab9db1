// Fused GaBP iteration, FP32, persistent blocks fed by TMA.
//
// Same per-tile work as the plain fused kernel (gabp_fused.cu): stage the 5 prior-message
// planes over the tile plus a 2-cell halo, compute the compensated beliefs of the tile plus a
// 1-cell halo, update the tile's cell factors and the observation factors based in the tile,
// write the damped messages to the other ping-pong buffer.  Here each block is persistent and
// walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... (row-major tile order, so the tiles in
// flight at any moment are spatial neighbours and their halos are served by L2).  One thread
// issues, per tile, two TMA tensor loads into an S-stage shared-memory ring:
//   * the 5 planes as one 3-D box (2 (TX+4) floats x (TY+4) rows x 5 planes), out-of-grid
//     positions zero-filled by the TMA unit;
//   * the window of observation pointers (TX+8) x (TY+3) of the observations-by-base-cell index,
// and completion is tracked by one mbarrier per stage (complete_tx), so the loads of the next
// S-1 tiles are in flight while the current tile computes.  Every mbarrier wait is bounded: on
// timeout the kernel raises the error flag, waits (bounded) for its own outstanding copies and
// returns.
//
// Requirements (checked on the host): FP32 messages, nx a multiple of 4 (16-byte row pitch of
// the index, 16-byte aligned box starts).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "gabp_device.cuh"
#include "gabp_internal.h"

namespace gabp {

namespace {

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

template <int TX, int TY, int S, int NT> struct TmaLayout {
    static constexpr int RX = TX + 4, RY = TY + 4;   // staged message window (cells)
    static constexpr int BX = TX + 2, BY = TY + 2;   // belief window
    static constexpr int OX = TX + 8, OY = TY + 3;   // observation-pointer window
    static constexpr uint32_t plane_bytes = 5u * RY * RX * 8u;
    static constexpr uint32_t optr_bytes = (uint32_t)OX * OY * 4u;
    static constexpr size_t stage = a128(plane_bytes) + a128(optr_bytes);
    static constexpr size_t bel_off = S * stage;
    static constexpr size_t bar_off = a128(bel_off + sizeof(Belief<float>) * BX * BY);
    static constexpr size_t ints_off = bar_off + 8 * (S + 1);   // S stage barriers + 1 test barrier
    static constexpr size_t bytes = ints_off + sizeof(int) * (2 * (TY + 1) + 1);
    static_assert(2 * RX <= 256 && RY <= 256 && OX <= 256, "TMA box dimension above 256");
};

template <int TX, int TY, int S, int NT>
__global__ void __launch_bounds__(NT) k_fused_tma(const __grid_constant__ CUtensorMap mplanes,
                                                  const __grid_constant__ CUtensorMap moptr, DevProblem p,
                                                  int src, float beta) {
    using LY = TmaLayout<TX, TY, S, NT>;
    constexpr int RX = LY::RX, RY = LY::RY, BX = LY::BX, BY = LY::BY, OX = LY::OX;
    extern __shared__ __align__(128) unsigned char smem[];
    Belief<float> *sb = reinterpret_cast<Belief<float> *>(smem + LY::bel_off);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + LY::bar_off);
    int *rstart = reinterpret_cast<int *>(smem + LY::ints_off);
    int *rpre = rstart + (TY + 1);
    int *flag = rpre + (TY + 1);

    const int nx = p.nx, ny = p.ny;
    const int64_t n = p.n;
    const int ntx = (nx + TX - 1) / TX;
    const int ntiles = ntx * ((ny + TY - 1) / TY);
    const int G = gridDim.x;
    const int tid = threadIdx.x;
    float2 *Q = (float2 *)p.P[src ^ 1];
    const float *O = (const float *)p.O[src];
    float *OQ = (float *)p.O[src ^ 1];

    auto issue = [&](int stage, int tile) {
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        unsigned char *base = smem + stage * LY::stage;
        const uint32_t bar = smem_addr(&bars[stage]);
        mbar_expect_tx(bar, LY::plane_bytes + LY::optr_bytes);
        tma_load_3d(smem_addr(base), &mplanes, 2 * (x0 - 2), y0 - 2, 0, bar);
        tma_load_2d(smem_addr(base + a128(LY::plane_bytes)), &moptr, x0 - 4, y0 - 2, bar);
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
    for (;; ++it) {
        const int tile = blockIdx.x + it * G;
        if (tile >= ntiles) break;
        const int stage = it % S;
        const uint32_t parity = (uint32_t)((it / S) & 1);
        if (!mbar_wait(smem_addr(&bars[stage]), parity)) *flag = 1;
        __syncthreads();
        if (*flag) break;

        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        const float2 *sm = reinterpret_cast<const float2 *>(smem + stage * LY::stage);   // [5][RY][RX]
        const int *W = reinterpret_cast<const int *>(smem + stage * LY::stage + a128(LY::plane_bytes));
        // observation pointer of base cell (x, y) from the staged window (origin x0-4, y0-2)
        auto wptr = [&](int x, int y) { return W[(y - y0 + 2) * OX + (x - x0 + 4)]; };

        // observation ranges of the tile's own base cells, one per tile row
        if (tid <= TY) {
            const int r = tid, gy = y0 + r;
            int lo = 0, cnt = 0;
            if (r < TY && gy < ny) {
                lo = wptr(x0, gy);
                cnt = wptr(min(x0 + TX, nx - 1), gy) - lo;
                if (cnt < 0) cnt = 0;
            }
            rstart[r] = lo;
            rpre[r] = cnt;
        }

        // compensated beliefs over the tile plus a 1-cell halo
        for (int q = tid; q < BX * BY; q += NT) {
            const int ly = q / BX, lx = q - ly * BX;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
            const int rx = lx + 1, ry = ly + 1;
            float2 m = sm[(DIR_C * RY + ry) * RX + rx];
            CompSum<float> se(m.x), sl(m.y);
            if (gx > 0) { m = sm[(DIR_E * RY + ry) * RX + rx - 1]; se.add(m.x); sl.add(m.y); }
            if (gx < nx - 1) { m = sm[(DIR_W * RY + ry) * RX + rx + 1]; se.add(m.x); sl.add(m.y); }
            if (gy > 0) { m = sm[(DIR_N * RY + ry - 1) * RX + rx]; se.add(m.x); sl.add(m.y); }
            if (gy < ny - 1) { m = sm[(DIR_S * RY + ry + 1) * RX + rx]; se.add(m.x); sl.add(m.y); }
            if (p.m > 0) {
                // corner 0: base (gx, gy); 1: (gx-1, gy); 2: (gx, gy-1); 3: (gx-1, gy-1).
                // An end pointer beyond the last column reads the zero fill: the range is empty,
                // as it must be (no base cell in the last column).
                const int a0 = wptr(gx, gy), a1 = wptr(gx + 1, gy);
                for (int k = a0; k < a1; ++k) { se.add(O[8 * (int64_t)k + 0]); sl.add(O[8 * (int64_t)k + 4]); }
                if (gx > 0) {
                    const int b0 = wptr(gx - 1, gy);
                    for (int k = b0; k < a0; ++k) { se.add(O[8 * (int64_t)k + 1]); sl.add(O[8 * (int64_t)k + 5]); }
                }
                if (gy > 0) {
                    const int c0 = wptr(gx, gy - 1), c1 = wptr(gx + 1, gy - 1);
                    for (int k = c0; k < c1; ++k) { se.add(O[8 * (int64_t)k + 2]); sl.add(O[8 * (int64_t)k + 6]); }
                    if (gx > 0) {
                        const int d0 = wptr(gx - 1, gy - 1);
                        for (int k = d0; k < c0; ++k) { se.add(O[8 * (int64_t)k + 3]); sl.add(O[8 * (int64_t)k + 7]); }
                    }
                }
            }
            se.finish();
            sl.finish();
            Belief<float> b;
            b.ehi = se.hi; b.elo = se.lo; b.lhi = sl.hi; b.llo = sl.lo;
            sb[q] = b;
        }
        __syncthreads();
        if (p.m > 0 && tid == 0) {
            int acc = 0;
            for (int r = 0; r < TY; ++r) {
                const int c = rpre[r];
                rpre[r] = acc;
                acc += c;
            }
            rpre[TY] = acc;
        }

        // prior cell factors of the tile
        const float var_prior = (float)(1.0 / p.gamma);
        for (int q = tid; q < TX * TY; q += NT) {
            const int ty = q / TX, tx = q - ty * TX;
            const int gx = x0 + tx, gy = y0 + ty;
            if (gx >= nx || gy >= ny) continue;
            const int64_t c = (int64_t)gy * nx + gx;
            const int deg = grid_degree(gy, gx, nx, ny);
            const float a[5] = {(float)p.aC[deg], gx > 0 ? -1.f : 0.f, gx < nx - 1 ? -1.f : 0.f,
                                gy > 0 ? -1.f : 0.f, gy < ny - 1 ? -1.f : 0.f};
            const int bxs[5] = {tx + 1, tx, tx + 2, tx + 1, tx + 1};
            const int bys[5] = {ty + 1, ty + 1, ty + 1, ty, ty + 2};
            float2 own[5];
            float lam[5], eta[5];
#pragma unroll
            for (int u = 0; u < 5; ++u) {
                own[u] = sm[(u * RY + ty + 2) * RX + tx + 2];
                if (a[u] != 0.f) {
                    cavity(sb[bys[u] * BX + bxs[u]], own[u].x, own[u].y, eta[u], lam[u]);
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
                Q[u * n + c] = out;
            }
        }
        __syncthreads();   // rpre is final; every thread is done with this stage's planes

        // observation factors based in the tile
        if (p.m > 0) {
            const int total = rpre[TY];
            const float *Wt = (const float *)p.ow;
            const float *YV = (const float *)p.ovar;
            for (int q = tid; q < total; q += NT) {
                int r = 0;
                while (r + 1 < TY && rpre[r + 1] <= q) ++r;
                const int64_t k = rstart[r] + (q - rpre[r]);
                const int b = p.obase[k];
                const int by = b / nx, bx = b - by * nx;
                const int lx = bx - x0 + 1, ly = by - y0 + 1;
                const int bidx[4] = {ly * BX + lx, ly * BX + lx + 1, (ly + 1) * BX + lx, (ly + 1) * BX + lx + 1};
                const float4 w4 = *reinterpret_cast<const float4 *>(Wt + 4 * k);
                const float a[4] = {w4.x, w4.y, w4.z, w4.w};
                const float4 oe4 = *reinterpret_cast<const float4 *>(O + 8 * k);
                const float4 ol4 = *reinterpret_cast<const float4 *>(O + 8 * k + 4);
                const float oe[4] = {oe4.x, oe4.y, oe4.z, oe4.w};
                const float ol[4] = {ol4.x, ol4.y, ol4.z, ol4.w};
                float lam[4], eta[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) cavity(sb[bidx[u]], oe[u], ol[u], eta[u], lam[u]);
                float L[4], E[4];
                factor_messages<float, 4>(a, YV[2 * k + 1], YV[2 * k], lam, eta, L, E);
                float4 ne, nl;
                ne.x = damp(oe[0], E[0], beta); ne.y = damp(oe[1], E[1], beta);
                ne.z = damp(oe[2], E[2], beta); ne.w = damp(oe[3], E[3], beta);
                nl.x = damp(ol[0], L[0], beta); nl.y = damp(ol[1], L[1], beta);
                nl.z = damp(ol[2], L[2], beta); nl.w = damp(ol[3], L[3], beta);
                *reinterpret_cast<float4 *>(OQ + 8 * k) = ne;
                *reinterpret_cast<float4 *>(OQ + 8 * k + 4) = nl;
            }
        }
        __syncthreads();   // beliefs and ranges are reused by the next tile

        if (tid == 0) {
            const int t2 = blockIdx.x + (it + S) * G;
            if (t2 < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(stage, t2);
            }
        }
    }

    if (*flag) {
        if (tid == 0) {
            atomicExch(p.err, 1);
            // drain this block's outstanding copies (bounded)
            for (int j = it; j < it + S; ++j) {
                const int t = blockIdx.x + j * G;
                if (t >= ntiles) break;
                mbar_wait(smem_addr(&bars[j % S]), (uint32_t)((j / S) & 1));
            }
        }
        __syncthreads();
    }
}

template <int TX, int TY, int S, int NT>
cudaError_t launch_cfg(const DevProblem &p, const TmaMaps &maps, int src, double beta, cudaStream_t st) {
    using LY = TmaLayout<TX, TY, S, NT>;
    static int grid_cache = 0;
    static int configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(k_fused_tma<TX, TY, S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)LY::bytes);
        if (e != cudaSuccess) return e;
        int nsm = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_tma<TX, TY, S, NT>, NT, LY::bytes);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cache = nsm * per_sm;
        configured_dev = dev;
    }
    const int ntiles = ((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
    const int grid = ntiles < grid_cache ? ntiles : grid_cache;
    k_fused_tma<TX, TY, S, NT><<<grid, NT, LY::bytes, st>>>(maps.planes[src], maps.optr, p, src, (float)beta);
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

bool tma_shape_supported(int tx, int ty) {
    return (tx == 64 && ty == 16) || (tx == 32 && ty == 16) || (tx == 64 && ty == 8) || (tx == 32 && ty == 32);
}

bool tma_problem_supported(const DevProblem &p) { return p.prec == 0 && p.nx % 4 == 0 && p.nx >= 4; }

// Tensor maps of both message buffers (3-D: 2 nx floats x ny rows x 5 planes) and of the
// observation index (2-D: nx x ny int32 of optr[0..n)), with boxes for the tile shape.
cudaError_t make_tma_maps(const DevProblem &p, int tx, int ty, TmaMaps &maps) {
    maps.valid = false;
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
    cuuint32_t box[2] = {(cuuint32_t)(tx + 8), (cuuint32_t)(ty + 3)};
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
    if (tx == 64 && ty == 16) return TmaLayout<64, 16, 2, 512>::bytes;
    if (tx == 32 && ty == 16) return TmaLayout<32, 16, 3, 256>::bytes;
    if (tx == 64 && ty == 8) return TmaLayout<64, 8, 2, 256>::bytes;
    if (tx == 32 && ty == 32) return TmaLayout<32, 32, 2, 512>::bytes;
    return 0;
}

cudaError_t launch_tma_iteration(const DevProblem &p, const TmaMaps &maps, int src, double beta,
                                 cudaStream_t st) {
    if (!maps.valid) return cudaErrorInvalidValue;
    if (maps.tx == 64 && maps.ty == 16) return launch_cfg<64, 16, 2, 512>(p, maps, src, beta, st);
    if (maps.tx == 32 && maps.ty == 16) return launch_cfg<32, 16, 3, 256>(p, maps, src, beta, st);
    if (maps.tx == 64 && maps.ty == 8) return launch_cfg<64, 8, 2, 256>(p, maps, src, beta, st);
    if (maps.tx == 32 && maps.ty == 32) return launch_cfg<32, 32, 2, 512>(p, maps, src, beta, st);
    return cudaErrorInvalidValue;
}

}  // namespace gabp
