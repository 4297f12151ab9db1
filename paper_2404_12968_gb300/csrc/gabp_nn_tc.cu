// Forward convolutions of the warm-start network on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), fed by TMA.
//
// A convolution out[p][co] = sum_{t, ci} in[p + d_t][ci] w[co][t][ci] is an implicit GEMM with
// M = pixels, N = output channels, K = taps x input channels.  A block computes tiles of
// 16 x 8 output pixels (M = 128, GEMM row m = 8 y + x) times N output channels:
//
//   * the input tile plus a one-pixel halo, 18 x 10 pixels, is loaded by TMA once per block of
//     16 input channels, as two [18][10][8] BF16 chunks (zero fill outside the image is the
//     convolution's zero padding).  Every tap (dy, dx) is then the same shared-memory matrix at
//     another start address: start + ((dy + 1) * 10 + (dx + 1)) * 16 bytes, 16 bytes between
//     the 8 pixels of a row, 160 bytes between pixel rows, one chunk pitch between the two
//     8-channel halves of K.  No input pixel is copied more than once per channel block.
//   * the weights of that channel block are a prepacked [tap][8-channel half][N][8] BF16 slab
//     (one bulk copy), the K-major canonical layout of the MMA's B operand.
//   * one MMA per tap (K = 16) accumulates into one of two TMEM accumulators of N FP32
//     columns, so the epilogue of one tile overlaps the MMAs of the next.
//
// Warp roles (192 threads): warp 4 issues the TMA copies into an S-stage mbarrier ring, one
// thread of warp 5 issues the MMAs and their commits, warps 0-3 (one TMEM lane quarter each)
// read the accumulators back (tcgen05.ld), add the bias, apply the activation and store BF16
// NHWC.  Optional fused epilogues: 2x2 average pooling, nearest upsampling plus a skip tensor
// (the decoder's 1x1 reductions), and the 1x1 FP32 head.  Every mbarrier wait is bounded; a
// wait that runs out raises the error flag and the block finishes without further copies.
//
// The weight gradient of training, dw[co][t][ci] = sum_p g[p][co] in[p + d_t][ci], is a GEMM
// with M = output channels, N = input channels and K = pixels, per tap (k_tc_wgrad).  Both
// operands come straight from the NHWC tensors: 8 channels of one pixel are 16 contiguous
// bytes, so a tile of 64 pixels (16 x 4) x 8 channels is one MN-major core-matrix column
// (8 pixels = 128 bytes per core matrix along K), loaded by one 5-D TMA copy per operand
// (channel-in-group, x, y, image, channel group) with zero fill outside the image for the tap
// shift.  One accumulator of N FP32 columns per block covers a chunk of pixel tiles; the
// epilogue writes it to a partial-sum buffer that a second kernel reduces in chunk order.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gabp_nn.h"

namespace gabp {
namespace nn {

namespace {

constexpr int TC_THREADS = 192;
constexpr int TILE_Y = 16, TILE_X = 8;          // output pixels per tile (M = 128)
constexpr int HALO_Y = TILE_Y + 2, HALO_X = TILE_X + 2;
constexpr uint32_t CHUNK_BYTES = HALO_Y * HALO_X * 16;   // one 8-channel halo chunk (2880 B)
constexpr uint32_t CHUNK_PITCH = 2944;                   // chunk pitch in shared memory (128-aligned)
constexpr uint32_t HALO_BYTES = 2 * CHUNK_PITCH;          // 16 channels

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// bounded wait for the phase with the given parity; false if it did not complete in time
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
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
        if (clock64() - t0 > (1LL << 32)) return false;
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor of tcgen05 (no swizzle, K-major canonical layout): start
// address, leading-dimension byte offset (between the 8-element K chunks), stride byte offset
// (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both MN-major (transpose bits 15
// and 16), M = 128, N.
__device__ __forceinline__ uint32_t instr_desc_mn(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N.
template <int N> __device__ __forceinline__ uint32_t instr_desc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void store16_bf16(__nv_bfloat16 *dst, const __nv_bfloat16 (&v)[16]) {
    uint4 q[2];
    __nv_bfloat16 *h = reinterpret_cast<__nv_bfloat16 *>(q);
#pragma unroll
    for (int j = 0; j < 16; ++j) h[j] = v[j];
    reinterpret_cast<uint4 *>(dst)[0] = q[0];
    reinterpret_cast<uint4 *>(dst)[1] = q[1];
}

template <int N, int T>
__global__ void __launch_bounds__(TC_THREADS) k_tc_conv(const __grid_constant__ CUtensorMap in_map, TcConvArgs a) {
    constexpr uint32_t WBYTES = (uint32_t)T * 32 * N;          // weight slab of one channel block
    extern __shared__ __align__(1024) unsigned char smem[];
    const int S = a.stages;
    const int nkb = a.Cin / 16;
    // resident weights: all nkb slabs stay in shared memory and the ring carries halos only;
    // otherwise every stage carries a halo and its weight slab
    const bool resident = a.resident != 0;
    const uint32_t wres = resident ? (uint32_t)nkb * WBYTES : 0u;   // resident weight bytes
    const uint32_t STAGE = resident ? HALO_BYTES : HALO_BYTES + WBYTES;   // multiples of 128
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + wres + (size_t)S * STAGE);
    // full[S], empty[S], acc_full[2], acc_empty[2], weights
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * S + 5);
    volatile int *fail = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = saddr(smem);
    auto full = [&](int s) { return saddr(&bars[s]); };
    auto empty = [&](int s) { return saddr(&bars[S + s]); };
    auto accf = [&](int i) { return saddr(&bars[2 * S + i]); };
    auto acce = [&](int i) { return saddr(&bars[2 * S + 2 + i]); };
    const uint32_t wbar = saddr(&bars[2 * S + 4]);
    const uint32_t ring = sbase + wres;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(accf(i), 1);
            mbar_init(acce(i), 4);
        }
        mbar_init(wbar, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                     "r"(2 * N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const int64_t ntiles = a.ntiles;
    auto tile_coords = [&](int64_t tile, int &b, int &y0, int &x0, int &nb) {
        nb = (int)(tile % a.nblocks);
        int64_t r = tile / a.nblocks;
        const int tx = (int)(r % a.tiles_x);
        r /= a.tiles_x;
        const int ty = (int)(r % a.tiles_y);
        b = (int)(r / a.tiles_y);
        y0 = ty * TILE_Y;
        x0 = tx * TILE_X;
    };

    if (warp == 4) {
        // ---- TMA producer ----
        if (lane == 0) {
            if (resident) {   // one output-channel block: load all its weight slabs once
                mbar_expect_tx(wbar, wres);
                for (int kb = 0; kb < nkb; ++kb)
                    bulk_load(sbase + (uint32_t)kb * WBYTES, a.wpk + (int64_t)kb * (WBYTES / 2), WBYTES, wbar);
            }
            int64_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && !*fail; tile += gridDim.x) {
                int b, y0, x0, nb;
                tile_coords(tile, b, y0, x0, nb);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t use = (uint32_t)(it / S);
                    if (!mbar_wait(empty(s), (use & 1) ^ 1)) {
                        *fail = 1;
                        break;
                    }
                    const uint32_t st = ring + (uint32_t)s * STAGE;
                    mbar_expect_tx(full(s), 2 * CHUNK_BYTES + (resident ? 0u : WBYTES));
                    tma_load_4d(st, &in_map, 16 * kb, x0 - 1, y0 - 1, b, full(s));
                    tma_load_4d(st + CHUNK_PITCH, &in_map, 16 * kb + 8, x0 - 1, y0 - 1, b, full(s));
                    if (!resident)
                        bulk_load(st + HALO_BYTES, a.wpk + ((int64_t)nb * nkb + kb) * (WBYTES / 2), WBYTES, full(s));
                }
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t idesc = instr_desc<N>();
            int64_t it = 0;
            int lt = 0;
            if (resident && !mbar_wait(wbar, 0)) *fail = 1;
            for (int64_t tile = blockIdx.x; tile < ntiles && !*fail; tile += gridDim.x, ++lt) {
                const int acc = lt & 1;
                if (!mbar_wait(acce(acc), (((uint32_t)lt >> 1) & 1) ^ 1)) {
                    *fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * N);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % S);
                    if (!mbar_wait(full(s), (uint32_t)(it / S) & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st = ring + (uint32_t)s * STAGE;
                    const uint32_t wsl = resident ? sbase + (uint32_t)kb * WBYTES : st + HALO_BYTES;
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const int dy = T == 9 ? t / 3 - 1 : 0, dx = T == 9 ? t % 3 - 1 : 0;
                        const uint64_t ad =
                            smem_desc(st + (uint32_t)(((dy + 1) * HALO_X + (dx + 1)) * 16), CHUNK_PITCH, HALO_X * 16);
                        const uint64_t bd = smem_desc(wsl + (uint32_t)(t * 2 * N * 16), N * 16, 128);
                        umma(d, ad, bd, idesc, (kb > 0 || t > 0) ? 1u : 0u);
                    }
                    umma_commit(empty(s));   // the stage is free once these MMAs have read it
                }
                if (!ok) {
                    *fail = 1;
                    break;
                }
                umma_commit(accf(acc));   // accumulator complete
            }
        }
    } else {
        // ---- epilogue: warps 0-3, TMEM lanes 32 w .. 32 w + 31 = tile pixels ----
        const int m = 32 * warp + lane;
        const int yy = m >> 3, xx = m & 7;
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            const bool ok = mbar_wait(accf(acc), ((uint32_t)lt >> 1) & 1);
            if (!ok) *fail = 1;
            if (__any_sync(0xffffffffu, !ok) || *fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int b, y0, x0, nb;
            tile_coords(tile, b, y0, x0, nb);
            const int gy = y0 + yy, gx = x0 + xx;
            const bool valid = gy < a.H && gx < a.W;
            const int co0 = nb * N;
            const int64_t pix = ((int64_t)b * a.H + gy) * a.W + gx;
            float h0 = 0.f, h1 = 0.f;
            if (a.head_w) {
                h0 = a.head_b[0];
                h1 = a.head_b[1];
            }
#pragma unroll 1
            for (int c = 0; c < N; c += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * N + c), r);
                __nv_bfloat16 v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float f = __uint_as_float(r[j]) + a.bias[co0 + c + j];
                    if (a.relu) f = fmaxf(f, 0.f);
                    v[j] = __float2bfloat16(f);
                }
                if (a.out && valid) store16_bf16(a.out + pix * a.Cout + co0 + c, v);
                if (a.pool_out) {
                    // 2x2 average: (y, x), (y, x+1), (y+1, x), (y+1, x+1) are lanes +0, +1, +8, +9
                    __nv_bfloat16 pv[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float f = __bfloat162float(v[j]);
                        const float f1 = __shfl_down_sync(0xffffffffu, f, 1);
                        const float f8 = __shfl_down_sync(0xffffffffu, f, 8);
                        const float f9 = __shfl_down_sync(0xffffffffu, f, 9);
                        pv[j] = __float2bfloat16(0.25f * (((f + f1) + f8) + f9));
                    }
                    if (valid && !(xx & 1) && !(yy & 1)) {
                        const int64_t q = ((int64_t)b * (a.H / 2) + gy / 2) * (a.W / 2) + gx / 2;
                        store16_bf16(a.pool_out + q * a.Cout + co0 + c, pv);
                    }
                }
                if (a.up_out && valid) {
                    // nearest upsampling to (2H, 2W) plus the skip tensor there
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int fy = 2 * gy + (q >> 1), fx = 2 * gx + (q & 1);
                        const int64_t fp = ((int64_t)b * (2 * a.H) + fy) * (2 * a.W) + fx;
                        const __nv_bfloat16 *sk = a.up_skip + fp * a.Cout + co0 + c;
                        uint4 sq[2];
                        sq[0] = reinterpret_cast<const uint4 *>(sk)[0];
                        sq[1] = reinterpret_cast<const uint4 *>(sk)[1];
                        const __nv_bfloat16 *sh = reinterpret_cast<const __nv_bfloat16 *>(sq);
                        __nv_bfloat16 u[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) u[j] = __float2bfloat16(__bfloat162float(v[j]) + __bfloat162float(sh[j]));
                        store16_bf16(a.up_out + fp * a.Cout + co0 + c, u);
                    }
                }
                if (a.head_w) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float f = __bfloat162float(v[j]);
                        h0 = fmaf(a.head_w[c + j], f, h0);
                        h1 = fmaf(a.head_w[a.Cout + c + j], f, h1);
                    }
                }
            }
            if (a.head_w && valid) {
                a.head_out[2 * pix] = h0;
                a.head_out[2 * pix + 1] = h1;
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce(acc));
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*fail && tid == 0) atomicExch(a.err, 1);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * N));
    }
}

// ---- weight gradient ----
constexpr int WG_THREADS = 192;
constexpr int WG_KX = 16;                               // pixels per tile row (one MMA, K = 16)

// Block: a group of taps [t0, t0 + tpc), output-channel block mb (128), input-channel block nb
// (N), pixel-tile chunk.  A tile is 16 x KY pixels.  Shared memory per stage:
//   A [16 groups][KY][16][8]: g at the tile's pixels, 8 output channels per group;
//   B [N / 8 groups][KY + 2 h][16 + 2 h][8]: the input at the tile's pixels plus a one-pixel
//     halo (h = 1 for 3x3 taps), so that every tap (dy, dx) of a tile row is the same matrix at
//     another start address, ((row + h + dy) (16 + 2 h) + h + dx) 16 bytes.
// Canonical MN-major, no swizzle: core matrix = 8 pixels x 8 channels (128 B), K-direction core
// matrices 128 B apart (LBO), channel-direction one group apart (SBO).  One MMA per tile row and
// tap accumulates into that tap's N TMEM columns.  Only the A groups of existing output channels
// are copied (a.ga of them); the rest of A is zeroed once and stays zero.
__global__ void __launch_bounds__(WG_THREADS) k_tc_wgrad(const __grid_constant__ CUtensorMap gmap,
                                                         const __grid_constant__ CUtensorMap xmap, TcWgradArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int S = a.stages, N = a.N, KY = a.ky, h = a.T == 9 ? 1 : 0;
    const int HX = WG_KX + 2 * h, HY = KY + 2 * h;
    const uint32_t AG = (uint32_t)(WG_KX * KY * 16), BG = (uint32_t)(HX * HY * 16);
    const uint32_t ABYTES = 16 * AG;
    const uint32_t STAGE = (ABYTES + (uint32_t)(N / 8) * BG + 127u) & ~127u;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)S * STAGE);   // full[S], empty[S], acc
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * S + 1);
    volatile int *fail = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = saddr(smem);
    auto full = [&](int s) { return saddr(&bars[s]); };
    auto empty = [&](int s) { return saddr(&bars[S + s]); };
    const uint32_t accb = saddr(&bars[2 * S]);
    const uint32_t need = (uint32_t)(a.tpc * N);
    const uint32_t tcols = need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : (need <= 256 ? 256u : 512u)));

    // block -> (chunk, tap group, mb, nb)
    int64_t r = blockIdx.x;
    const int nb = (int)(r % a.nbn);
    r /= a.nbn;
    const int mb = (int)(r % a.nbm);
    r /= a.nbm;
    const int tg = (int)(r % a.ngroups);
    const int chunk = (int)(r / a.ngroups);
    const int t0 = tg * a.tpc;
    const int ntap = a.T - t0 < a.tpc ? a.T - t0 : a.tpc;
    const int64_t kt0 = (int64_t)chunk * a.per_chunk;
    const int64_t kt1 = kt0 + a.per_chunk < a.ktiles ? kt0 + a.per_chunk : a.ktiles;
    const int nk = (int)(kt1 > kt0 ? kt1 - kt0 : 0);

    // A rows past the copied groups: zero, written once through the generic proxy and made
    // visible to the tensor core's (async proxy) reads
    if (a.ga < 16) {
        const uint32_t zbytes = (16u - (uint32_t)a.ga) * AG;
        for (int s = 0; s < S; ++s) {
            uint4 *z = reinterpret_cast<uint4 *>(smem + (size_t)s * STAGE + (size_t)a.ga * AG);
            for (uint32_t i = tid; i < zbytes / 16; i += WG_THREADS) z[i] = make_uint4(0, 0, 0, 0);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(accb, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 4) {
        // ---- TMA producer: tile k = (image, tile row, tile column) ----
        if (lane == 0) {
            for (int i = 0; i < nk && !*fail; ++i) {
                const int s = i % S;
                if (!mbar_wait(empty(s), ((uint32_t)(i / S) & 1) ^ 1)) {
                    *fail = 1;
                    break;
                }
                const int64_t k = kt0 + i;
                const int tx = (int)(k % a.tiles_x);
                const int64_t q = k / a.tiles_x;
                const int ty = (int)(q % a.tiles_y);
                const int b = (int)(q / a.tiles_y);
                const int x0 = tx * WG_KX, y0 = ty * KY;
                const uint32_t st = sbase + (uint32_t)s * STAGE;
                mbar_expect_tx(full(s), (uint32_t)a.ga * AG + (uint32_t)(N / 8) * BG);
                tma_load_5d(st, &gmap, 0, x0, y0, b, 16 * mb, full(s));
                tma_load_5d(st + ABYTES, &xmap, 0, x0 - h, y0 - h, b, nb * (N / 8), full(s));
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer: one MMA (K = 16) per tile row and tap ----
        if (lane == 0) {
            const uint32_t idesc = instr_desc_mn(N);
            bool ok = true;
            for (int i = 0; i < nk && !*fail; ++i) {
                const int s = i % S;
                if (!mbar_wait(full(s), (uint32_t)(i / S) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = sbase + (uint32_t)s * STAGE;
                for (int j = 0; j < ntap; ++j) {
                    const int t = t0 + j;
                    const int dy = a.T == 9 ? t / 3 - 1 : 0, dx = a.T == 9 ? t % 3 - 1 : 0;
                    for (int kk = 0; kk < KY; ++kk) {
                        const uint64_t ad = smem_desc(st + (uint32_t)kk * 256u, 128u, AG);
                        const uint64_t bd =
                            smem_desc(st + ABYTES + (uint32_t)(((kk + h + dy) * HX + h + dx) * 16), 128u, BG);
                        umma(tmem + (uint32_t)(j * N), ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                umma_commit(empty(s));   // the stage is free once these MMAs have read it
            }
            if (!ok) *fail = 1;
            umma_commit(accb);   // also after a failure, so that the epilogue does not wait out
        }
    } else {
        // ---- epilogue: warps 0-3, TMEM lane 32 w + lane = output channel 128 mb + 32 w + lane ----
        const bool ok = mbar_wait(accb, 0);
        if (!ok) *fail = 1;
        // warp-uniform decision: tcgen05.ld is a whole-warp instruction
        const bool go = __all_sync(0xffffffffu, ok && !*fail);
        const int co = 128 * mb + 32 * warp + lane;
        if (go && nk > 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int j = 0; j < ntap; ++j) {
                float *dst = a.part + (((int64_t)chunk * a.Cout + co) * a.T + t0 + j) * a.Cin + nb * N;
#pragma unroll 1
                for (int c = 0; c < N; c += 16) {
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(j * N + c), v);
                    if (co < a.Cout) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            *reinterpret_cast<float4 *>(dst + c + e) =
                                make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                                            __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
                    }
                }
            }
        } else if (go && co < a.Cout) {   // an empty chunk: zero partial sums
            for (int j = 0; j < ntap; ++j) {
                float *dst = a.part + (((int64_t)chunk * a.Cout + co) * a.T + t0 + j) * a.Cin + nb * N;
                for (int c = 0; c < N; ++c) dst[c] = 0.f;
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*fail && tid == 0) atomicExch(a.err, 1);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
    }
}

// packed[nb][kb][t][h][n][e] = w[nb * N + n][t][16 kb + 8 h + e]
__global__ void k_tc_pack(const __nv_bfloat16 *w, int Cout, int T, int Cin, int N, __nv_bfloat16 *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)Cout * T * Cin;
    if (i >= total) return;
    const int e = (int)(i & 7);
    int64_t r = i >> 3;
    const int n = (int)(r % N);
    r /= N;
    const int h = (int)(r & 1);
    r >>= 1;
    const int t = (int)(r % T);
    r /= T;
    const int nkb = Cin / 16;
    const int kb = (int)(r % nkb);
    const int nb = (int)(r / nkb);
    out[i] = w[((int64_t)(nb * N + n) * T + t) * Cin + 16 * kb + 8 * h + e];
}

PFN_cuTensorMapEncodeTiled_v12000 tc_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    return fn;
}

template <int N, int T>
cudaError_t tc_launch(const CUtensorMap &map, TcConvArgs a, cudaStream_t st) {
    static int configured_dev = -1;
    static int nsm = 0, occ_threads = 0;
    const uint32_t wbytes = (uint32_t)T * 32 * N;
    const int nkb = a.Cin / 16;
    const uint32_t wall = (uint32_t)nkb * wbytes;
    a.resident = (a.nblocks == 1 && wall <= 48u * 1024u) ? 1 : 0;
    size_t smem;
    if (a.resident) {
        int S = (int)((96u * 1024u - wall) / HALO_BYTES);
        a.stages = S < 2 ? 2 : (S > 8 ? 8 : S);
        smem = wall + (size_t)a.stages * HALO_BYTES;
    } else {
        const uint32_t stage = HALO_BYTES + wbytes;
        int S = (int)((72u * 1024u) / stage);
        a.stages = S < 2 ? 2 : (S > 4 ? 4 : S);
        smem = (size_t)a.stages * stage;
    }
    smem += 8 * (2 * a.stages + 5) + 16;
    // blocks per SM: registers and threads (occupancy without shared memory), shared memory
    // (228 KB, 1 KB reserved per block) and tensor memory (512 columns, 2N per block); the
    // shared-memory request is raised so that the SM cannot host more blocks than its tensor
    // memory holds
    const int tmem_cap = 512 / (2 * N);
    const size_t smem_floor = (size_t)(227 * 1024) / (size_t)(tmem_cap + 1) + 1024;
    if (smem < smem_floor) smem = smem_floor;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(k_tc_conv<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        // registers and threads per SM from the kernel's attributes
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_tc_conv<N, T>);
        if (e != cudaSuccess) return e;
        const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
        occ_threads = 65536 / (regs_warp * (TC_THREADS / 32));
        if (occ_threads > 2048 / TC_THREADS) occ_threads = 2048 / TC_THREADS;
        configured_dev = dev;
    }
    int per_sm = (int)((228 * 1024) / (smem + 1024));
    if (per_sm > occ_threads) per_sm = occ_threads;
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > a.ntiles) grid = a.ntiles;
    k_tc_conv<N, T><<<(unsigned)grid, TC_THREADS, smem, st>>>(map, a);
    return cudaGetLastError();
}

bool encode_nhwc_groups(CUtensorMap &map, const __nv_bfloat16 *p, int B, int H, int W, int C, int bx, int by,
                        int groups_box) {
    auto enc = tc_encoder();
    if (!enc) return false;
    // [B][H][W][C] viewed as (channel in group, x, y, image, 8-channel group)
    cuuint64_t dims[5] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B, (cuuint64_t)(C / 8)};
    cuuint64_t strides[4] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2, 16};
    cuuint32_t box[5] = {8, (cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)groups_box};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void *)p, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_block_n(int Cout) { return Cout < 128 ? Cout : 128; }

cudaError_t tc_wgrad(TcWgradArgs a, float *dw, cudaStream_t st) {
    if (a.Cin % 16 || a.Cout % 8 || a.Cin < 16 || (a.T != 1 && a.T != 9) || a.B < 1 || a.H < 1 || a.W < 1)
        return cudaErrorInvalidValue;
    a.N = a.Cin <= 256 ? a.Cin : 256;
    if (a.Cin % a.N) return cudaErrorInvalidValue;
    a.nbn = a.Cin / a.N;
    a.nbm = (a.Cout + 127) / 128;
    a.ga = a.Cout / 8 < 16 ? a.Cout / 8 : 16;
    // taps per block: as many N-column accumulators as the 512 TMEM columns hold, in groups of
    // balanced size
    const int maxt = 512 / a.N;
    a.ngroups = (a.T + maxt - 1) / maxt;
    a.tpc = (a.T + a.ngroups - 1) / a.ngroups;
    const int h = a.T == 9 ? 1 : 0;
    // tile height: 8 pixel rows when three stages of it fit in shared memory, else 4
    auto stage_bytes = [&](int ky) {
        const uint32_t ab = 16u * WG_KX * ky * 16, bb = (uint32_t)(a.N / 8) * (WG_KX + 2 * h) * (ky + 2 * h) * 16;
        return (ab + bb + 127u) & ~127u;
    };
    a.ky = stage_bytes(8) * 3 <= 196u * 1024u ? 8 : 4;
    const uint32_t stage = stage_bytes(a.ky);
    int S = (int)((196u * 1024u) / stage);
    a.stages = S > 6 ? 6 : S;
    if (a.stages < 2) return cudaErrorInvalidConfiguration;
    a.tiles_x = (a.W + WG_KX - 1) / WG_KX;
    a.tiles_y = (a.H + a.ky - 1) / a.ky;
    a.ktiles = (int64_t)a.B * a.tiles_y * a.tiles_x;
    static int configured_dev = -1, nsm = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(k_tc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    // blocks: about one per SM per resident slot over (chunk, tap group, output block, input
    // block); every chunk's partial sums must fit the buffer
    const int64_t per_chunk_blocks = (int64_t)a.ngroups * a.nbm * a.nbn;
    const int64_t count = (int64_t)a.Cout * a.T * a.Cin;
    const int resident = a.tpc * a.N <= 256 && stage * a.stages <= 100u * 1024u ? 2 : 1;
    int64_t chunks = ((int64_t)resident * nsm + per_chunk_blocks - 1) / per_chunk_blocks;
    if (chunks > a.ktiles) chunks = a.ktiles;
    if (chunks * count > a.part_cap) chunks = a.part_cap / count;
    if (chunks < 1) return cudaErrorInvalidValue;
    a.per_chunk = (a.ktiles + chunks - 1) / chunks;
    a.chunks = (int)((a.ktiles + a.per_chunk - 1) / a.per_chunk);
    const size_t smem = (size_t)a.stages * stage + 8 * (2 * a.stages + 1) + 16;
    CUtensorMap gmap, xmap;
    if (!encode_nhwc_groups(gmap, a.g, a.B, a.H, a.W, a.Cout, WG_KX, a.ky, a.ga) ||
        !encode_nhwc_groups(xmap, a.in, a.B, a.H, a.W, a.Cin, WG_KX + 2 * h, a.ky + 2 * h, a.N / 8))
        return cudaErrorInvalidValue;
    const int64_t grid = (int64_t)a.chunks * per_chunk_blocks;
    k_tc_wgrad<<<(unsigned)grid, WG_THREADS, smem, st>>>(gmap, xmap, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_chunks(a.part, a.chunks, count, dw, st);
}

cudaError_t tc_pack_weights(const __nv_bfloat16 *w, int Cout, int T, int Cin, __nv_bfloat16 *out, cudaStream_t st) {
    const int64_t total = (int64_t)Cout * T * Cin;
    k_tc_pack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(w, Cout, T, Cin, tc_block_n(Cout), out);
    return cudaGetLastError();
}

cudaError_t tc_conv(const __nv_bfloat16 *in, TcConvArgs a, cudaStream_t st) {
    const int N = tc_block_n(a.Cout);
    if ((a.T != 1 && a.T != 9) || a.Cin % 16 || a.Cout % N || (N != 32 && N != 64 && N != 128) || a.W < 1 ||
        a.H < 1 || a.B < 1)
        return cudaErrorInvalidValue;
    if (a.pool_out && (a.H % 2 || a.W % 2)) return cudaErrorInvalidValue;
    if (a.up_out && !a.up_skip) return cudaErrorInvalidValue;
    if (a.head_w && a.Cout != 32) return cudaErrorInvalidValue;
    auto enc = tc_encoder();
    if (!enc) return cudaErrorNotSupported;
    // activation tensor [B][H][W][Cin] BF16, box of 8 channels x 10 x 18 pixels x 1 image
    CUtensorMap map;
    cuuint64_t dims[4] = {(cuuint64_t)a.Cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.B};
    cuuint64_t strides[3] = {(cuuint64_t)a.Cin * 2, (cuuint64_t)a.W * a.Cin * 2, (cuuint64_t)a.H * a.W * a.Cin * 2};
    cuuint32_t box[4] = {8, HALO_X, HALO_Y, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)in, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    a.nblocks = a.Cout / N;
    a.tiles_x = (a.W + TILE_X - 1) / TILE_X;
    a.tiles_y = (a.H + TILE_Y - 1) / TILE_Y;
    a.ntiles = (int64_t)a.B * a.tiles_y * a.tiles_x * a.nblocks;
    if (N == 32) return a.T == 9 ? tc_launch<32, 9>(map, a, st) : tc_launch<32, 1>(map, a, st);
    if (N == 64) return a.T == 9 ? tc_launch<64, 9>(map, a, st) : tc_launch<64, 1>(map, a, st);
    return a.T == 9 ? tc_launch<128, 9>(map, a, st) : tc_launch<128, 1>(map, a, st);
}


}  // namespace nn
}  // namespace gabp
