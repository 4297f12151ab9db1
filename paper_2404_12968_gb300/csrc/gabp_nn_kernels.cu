// Kernels of the learned warm start's convolutional network: BF16 tensor-core convolutions
// with FP32 accumulation (forward and backward), and the small element-wise kernels around
// them.  Activations are NHWC BF16 ([B][H][W][C], channels contiguous); weights are
// [Cout][T][Cin] BF16 with T = 9 taps (3x3, zero padding 1) or T = 1 (1x1).
//
// Convolution as an implicit GEMM: out[p][co] = sum_{t, ci} in[p + d_t][ci] * w[co][t][ci], with
// M = pixels, N = output channels, K = taps x input channels.  Tiles of A (shifted input pixels)
// and B (weights) are staged in shared memory with cp.async (zero-filled outside the image),
// double buffered, and multiplied with mma.sync m16n8k16 BF16 -> FP32 fragments loaded by
// ldmatrix.  The backward pass w.r.t. the input is the same kernel on flipped, transposed
// weights; the backward pass w.r.t. the weights is a GEMM over pixels (split into chunks whose
// FP32 partial sums are reduced in a fixed order).
#include <cuda_bf16.h>
#include <stdint.h>

#include "gabp_nn.h"

namespace gabp {
namespace nn {

namespace {

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    // 16-byte async copy; src-size 0 zero-fills the destination
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t &r0, uint32_t &r1, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(saddr(p)));
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

constexpr int CT = 256;   // threads per convolution block
constexpr int BM = 128;   // pixels per block tile

// ---- forward / backward-data convolution ----
// BN output channels per block (32 or 64), BK input channels per k-step (16 or 32).
template <int BN, int BK>
__global__ void __launch_bounds__(CT) k_conv(ConvArgs a) {
    constexpr int AS = BK + 8;   // smem row stride (bf16), keeps ldmatrix rows on distinct banks
    __shared__ __align__(16) __nv_bfloat16 sA[2][BM * AS];
    __shared__ __align__(16) __nv_bfloat16 sB[2][BN * AS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;        // 4 warps along M (32 rows each), 2 along N
    constexpr int WN = BN / 2;                      // warp tile 32 x WN
    constexpr int NT = WN / 8;                      // n8 tiles per warp
    const int64_t P = (int64_t)a.B * a.H * a.W;
    const int64_t p0 = (int64_t)blockIdx.x * BM;
    const int co0 = blockIdx.y * BN;
    const int T = a.T, Cin = a.Cin;
    const int kc = Cin / BK;                        // channel blocks per tap
    const int nk = T * kc;

    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    constexpr int ACH = BK / 8;   // 16-byte chunks per pixel row
    auto load_tile = [&](int kt, int buf) {
        const int t = kt / kc, c0 = (kt - t * kc) * BK;
        const int dy = T == 9 ? t / 3 - 1 : 0, dx = T == 9 ? t % 3 - 1 : 0;
        for (int q = tid; q < BM * ACH; q += CT) {
            const int r = q / ACH, ch = q - r * ACH;
            const int64_t p = p0 + r;
            bool ok = p < P;
            const __nv_bfloat16 *src = a.in;
            if (ok) {
                const int64_t img = p / ((int64_t)a.H * a.W);
                const int rem = (int)(p - img * a.H * a.W);
                const int y = rem / a.W + dy, x = rem - (rem / a.W) * a.W + dx;
                ok = y >= 0 && y < a.H && x >= 0 && x < a.W;
                if (ok) src = a.in + ((img * a.H + y) * a.W + x) * Cin + c0 + ch * 8;
            }
            cp_async16(&sA[buf][r * AS + ch * 8], src, ok);
        }
        for (int q = tid; q < BN * ACH; q += CT) {
            const int r = q / ACH, ch = q - r * ACH;
            const __nv_bfloat16 *src = a.w + ((int64_t)(co0 + r) * T + t) * Cin + c0 + ch * 8;
            cp_async16(&sB[buf][r * AS + ch * 8], src, true);
        }
        cp_async_commit();
    };

    load_tile(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            load_tile(kt + 1, buf ^ 1);
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
#pragma unroll
        for (int k16 = 0; k16 < BK / 16; ++k16) {
            uint32_t af[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm * 32 + i * 16 + (lane & 15);
                const int col = k16 * 16 + (lane >> 4) * 8;
                ldsm_x4(af[i][0], af[i][1], af[i][2], af[i][3], &sA[buf][row * AS + col]);
            }
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                uint32_t b0, b1;
                const int nrow = wn * WN + j * 8 + (lane & 7);
                const int col = k16 * 16 + ((lane >> 3) & 1) * 8;
                ldsm_x2(b0, b1, &sB[buf][nrow * AS + col]);
#pragma unroll
                for (int i = 0; i < 2; ++i) mma16816(acc[i][j], af[i][0], af[i][1], af[i][2], af[i][3], b0, b1);
            }
        }
        __syncthreads();
    }

    // epilogue: + bias (+ skip), optional ReLU, store BF16 (or FP32)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t p = p0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
                if (p >= P) continue;
                const int co = co0 + wn * WN + j * 8 + (lane & 3) * 2;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if (a.bias) {
                    v0 += a.bias[co];
                    v1 += a.bias[co + 1];
                }
                if (a.skip) {
                    const __nv_bfloat162 s = *reinterpret_cast<const __nv_bfloat162 *>(a.skip + p * a.Cout + co);
                    v0 += __bfloat162float(s.x);
                    v1 += __bfloat162float(s.y);
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162 *>(a.out + p * a.Cout + co) = __floats2bfloat162_rn(v0, v1);
            }
}

// ---- backward w.r.t. the weights ----
// part[chunk][co][t][ci] = sum over the chunk's pixels p of g[p][co] * in[p + d_t][ci].
// Block tile 32 (co) x BNI (ci), one tap, one pixel chunk; k-steps of 32 pixels.
template <int BNI>
__global__ void __launch_bounds__(128) k_conv_wgrad(WgradArgs a) {
    constexpr int KP = 32;            // pixels per k-step
    constexpr int GS = 32 + 8;        // smem stride of the g tile (co)
    constexpr int XS = BNI + 8;       // smem stride of the input tile (ci)
    __shared__ __align__(16) __nv_bfloat16 sG[2][KP * GS];
    __shared__ __align__(16) __nv_bfloat16 sX[2][KP * XS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;      // 2 x 2 warps; warp tile 16 (co) x BNI/2 (ci)
    constexpr int WN = BNI / 2, NT = WN / 8;
    const int co0 = blockIdx.x * 32, ci0 = blockIdx.y * BNI;
    const int t = blockIdx.z % a.T, chunk = blockIdx.z / a.T;
    const int dy = a.T == 9 ? t / 3 - 1 : 0, dx = a.T == 9 ? t % 3 - 1 : 0;
    const int64_t P = (int64_t)a.B * a.H * a.W;
    const int64_t pb = (int64_t)chunk * a.chunk_pixels;
    const int64_t pe = pb + a.chunk_pixels < P ? pb + a.chunk_pixels : P;
    const int nk = (int)((pe - pb + KP - 1) / KP);

    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;

    auto load = [&](int kt, int buf) {
        const int64_t pk = pb + (int64_t)kt * KP;
        for (int q = tid; q < KP * 4; q += 128) {   // g tile: 32 pixels x 32 co = 4 chunks per pixel
            const int r = q >> 2, ch = q & 3;
            const int64_t p = pk + r;
            const bool ok = p < pe;
            cp_async16(&sG[buf][r * GS + ch * 8], ok ? a.g + p * a.Cout + co0 + ch * 8 : a.g, ok);
        }
        for (int q = tid; q < KP * (BNI / 8); q += 128) {
            const int r = q / (BNI / 8), ch = q - r * (BNI / 8);
            const int64_t p = pk + r;
            bool ok = p < pe;
            const __nv_bfloat16 *src = a.in;
            if (ok) {
                const int64_t img = p / ((int64_t)a.H * a.W);
                const int rem = (int)(p - img * a.H * a.W);
                const int y = rem / a.W + dy, x = rem - (rem / a.W) * a.W + dx;
                ok = y >= 0 && y < a.H && x >= 0 && x < a.W;
                if (ok) src = a.in + ((img * a.H + y) * a.W + x) * a.Cin + ci0 + ch * 8;
            }
            cp_async16(&sX[buf][r * XS + ch * 8], src, ok);
        }
        cp_async_commit();
    };

    if (nk > 0) load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            load(kt + 1, buf ^ 1);
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
#pragma unroll
        for (int k16 = 0; k16 < KP / 16; ++k16) {
            // A = g^T (co x pixels): stored [pixel][co], loaded transposed
            uint32_t a0, a1, a2, a3;
            {
                const int mat = lane >> 3, r8 = lane & 7;
                const int prow = k16 * 16 + (mat >> 1) * 8 + r8;
                const int ccol = wm * 16 + (mat & 1) * 8;
                ldsm_x4_t(a0, a1, a2, a3, &sG[buf][prow * GS + ccol]);
            }
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                uint32_t b0, b1;
                const int prow = k16 * 16 + ((lane >> 3) & 1) * 8 + (lane & 7);
                const int ccol = wn * WN + j * 8;
                ldsm_x2_t(b0, b1, &sX[buf][prow * XS + ccol]);
                mma16816(acc[j], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncthreads();
    }
    float *dst = a.part + (int64_t)chunk * a.Cout * a.T * a.Cin;
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co = co0 + wm * 16 + (lane >> 2) + h * 8;
            const int ci = ci0 + wn * WN + j * 8 + (lane & 3) * 2;
            dst[((int64_t)co * a.T + t) * a.Cin + ci] = acc[j][2 * h];
            dst[((int64_t)co * a.T + t) * a.Cin + ci + 1] = acc[j][2 * h + 1];
        }
}

// many chunks of few values: one block per value, the chunks strided over its threads, then a
// fixed-shape tree (a fixed order)
__global__ void k_reduce_chunks_wide(const float *part, int chunks, int64_t count, float *out) {
    __shared__ float sh[256];
    const int64_t i = blockIdx.x;
    float s = 0.f;
    for (int c = threadIdx.x; c < chunks; c += 256) s += part[(int64_t)c * count + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0];
}

// sum the chunk partials in chunk order
__global__ void k_reduce_chunks(const float *part, int chunks, int64_t count, float *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * count + i];
    out[i] = s;
}

// bias gradient, first stage: part[b][c] = sum of g[p][c] over the pixels of chunk b.  A block
// reads R = 256 / C pixels per step, C consecutive threads per pixel (coalesced), then adds its
// R row sums per channel in a fixed order.
__global__ void k_bias_part(const __nv_bfloat16 *g, int64_t P, int C, int64_t per_chunk, float *part) {
    __shared__ float sh[256];
    const int R = 256 / C;
    const int c = threadIdx.x % C, r = threadIdx.x / C;
    const int64_t p0 = (int64_t)blockIdx.x * per_chunk;
    const int64_t p1 = p0 + per_chunk < P ? p0 + per_chunk : P;
    float s = 0.f;
    if (r < R)
        for (int64_t p = p0 + r; p < p1; p += R) s += __bfloat162float(g[p * C + c]);
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int q = 0; q < R; ++q) t += sh[q * C + threadIdx.x];
        part[(int64_t)blockIdx.x * C + threadIdx.x] = t;
    }
}

// w_t[ci][t][co] = w[co][8 - t][ci] (3x3) or w[co][0][ci] (1x1): weights of the input gradient
__global__ void k_flip_transpose(const __nv_bfloat16 *w, int Cout, int T, int Cin, __nv_bfloat16 *wt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)Cout * T * Cin;
    if (i >= n) return;
    const int ci = (int)(i % Cin);
    const int t = (int)((i / Cin) % T);
    const int co = (int)(i / ((int64_t)Cin * T));
    wt[((int64_t)ci * T + (T - 1 - t)) * Cout + co] = w[i];
}

__global__ void k_relu_bwd(const __nv_bfloat16 *y, const __nv_bfloat16 *dy, __nv_bfloat16 *dx, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    dx[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16(0.f);
}

// 2x2 average pooling
__global__ void k_pool(const __nv_bfloat16 *x, int B, int H, int W, int C, __nv_bfloat16 *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    const int64_t n = (int64_t)B * Ho * Wo * C;
    if (i >= n) return;
    const int c = (int)(i % C);
    const int64_t q = i / C;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho);
    const int64_t b = q / ((int64_t)Wo * Ho);
    const __nv_bfloat16 *s = x + ((b * H + 2 * yo) * W + 2 * xo) * C + c;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[(int64_t)W * C]) +
                    __bfloat162float(s[(int64_t)W * C + C]);
    y[i] = __float2bfloat16(0.25f * v);
}

// backward of the pooling, accumulated into dx (dx += dy / 4 on each of the 4 pixels)
__global__ void k_pool_bwd_add(const __nv_bfloat16 *dy, int B, int H, int W, int C, __nv_bfloat16 *dx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)B * H * W * C;
    if (i >= n) return;
    const int c = (int)(i % C);
    const int64_t q = i / C;
    const int x = (int)(q % W), y = (int)((q / W) % H);
    const int64_t b = q / ((int64_t)W * H);
    const float g = __bfloat162float(dy[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]);
    dx[i] = __float2bfloat16(__bfloat162float(dx[i]) + 0.25f * g);
}

// y = nearest-upsample(r) + s   (r at half resolution)
__global__ void k_up_add(const __nv_bfloat16 *r, const __nv_bfloat16 *s, int B, int H, int W, int C, __nv_bfloat16 *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)B * H * W * C;
    if (i >= n) return;
    const int c = (int)(i % C);
    const int64_t q = i / C;
    const int x = (int)(q % W), yy = (int)((q / W) % H);
    const int64_t b = q / ((int64_t)W * H);
    y[i] = __float2bfloat16(__bfloat162float(r[((b * (H / 2) + yy / 2) * (W / 2) + x / 2) * C + c]) +
                            __bfloat162float(s[i]));
}

// dr = sum over each 2x2 block of dy (backward of the nearest upsampling)
__global__ void k_down_sum(const __nv_bfloat16 *dy, int B, int H, int W, int C, __nv_bfloat16 *dr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    const int64_t n = (int64_t)B * Ho * Wo * C;
    if (i >= n) return;
    const int c = (int)(i % C);
    const int64_t q = i / C;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho);
    const int64_t b = q / ((int64_t)Wo * Ho);
    const __nv_bfloat16 *s = dy + ((b * H + 2 * yo) * W + 2 * xo) * C + c;
    dr[i] = __float2bfloat16(__bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[(int64_t)W * C]) +
                             __bfloat162float(s[(int64_t)W * C + C]));
}

__global__ void k_add(const __nv_bfloat16 *a, __nv_bfloat16 *b, int64_t n) {   // b += a
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// head: out[p][j] = sum_c w[j][c] x[p][c] + b[j], j < 2 (FP32 out)
__global__ void k_head(const __nv_bfloat16 *x, int64_t P, int C, const float *w, const float *b, float *out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    float s0 = b[0], s1 = b[1];
    for (int c = 0; c < C; ++c) {
        const float v = __bfloat162float(x[p * C + c]);
        s0 = fmaf(w[c], v, s0);
        s1 = fmaf(w[C + c], v, s1);
    }
    out[2 * p] = s0;
    out[2 * p + 1] = s1;
}

// loss = mean over pixels of (o0 - t0)^2 + (o1 - t1)^2; d out = 2 (o - t) / P; block partials
__global__ void k_loss(const float *out, const float *target, int64_t P, float *dout, float *part) {
    __shared__ float sh[256];
    float s = 0.f;
    const float inv = 1.f / (float)P;
    for (int64_t p = blockIdx.x * 256 + threadIdx.x; p < P; p += (int64_t)gridDim.x * 256) {
        const float e0 = out[2 * p] - target[2 * p], e1 = out[2 * p + 1] - target[2 * p + 1];
        s += e0 * e0 + e1 * e1;
        dout[2 * p] = 2.f * e0 * inv;
        dout[2 * p + 1] = 2.f * e1 * inv;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0] * inv;
}

// head backward: dx[p][c] = sum_j dout[p][j] w[j][c] (BF16 out); dw, db by chunked partial sums
__global__ void k_head_bwd_x(const float *dout, int64_t P, int C, const float *w, __nv_bfloat16 *dx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= P * C) return;
    const int64_t p = i / C;
    const int c = (int)(i - p * C);
    dx[i] = __float2bfloat16(dout[2 * p] * w[c] + dout[2 * p + 1] * w[C + c]);
}

__global__ void k_head_bwd_w(const float *dout, const __nv_bfloat16 *x, int64_t P, int C, float *part) {
    // part[block][2*C + 2]: per block sums of dout[p][j] x[p][c] and dout[p][j]
    extern __shared__ float sh2[];
    const int K = 2 * C + 2;
    for (int k = threadIdx.x; k < K; k += blockDim.x) sh2[k] = 0.f;
    __syncthreads();
    const int64_t p0 = (int64_t)blockIdx.x * 1024;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float s = 0.f;
        for (int64_t p = p0; p < p0 + 1024 && p < P; ++p) {
            if (k < 2 * C) s += dout[2 * p + k / C] * __bfloat162float(x[p * C + (k % C)]);
            else s += dout[2 * p + (k - 2 * C)];
        }
        part[(int64_t)blockIdx.x * K + k] = s;
    }
}

// Adam (decoupled from the BF16 copy): FP32 master weights w, moments m, v; w16 = bf16(w)
__global__ void k_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16 *w16) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float *x, __nv_bfloat16 *y, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t conv(const ConvArgs &a, cudaStream_t st) {
    if (a.Cout % 32 || (a.Cin % 16) || (a.T != 1 && a.T != 9)) return cudaErrorInvalidValue;
    const int64_t P = (int64_t)a.B * a.H * a.W;
    const bool bn64 = a.Cout % 64 == 0;
    const bool bk32 = a.Cin % 32 == 0;
    dim3 grid((unsigned)((P + BM - 1) / BM), (unsigned)(a.Cout / (bn64 ? 64 : 32)));
    if (bn64 && bk32) k_conv<64, 32><<<grid, CT, 0, st>>>(a);
    else if (bn64) k_conv<64, 16><<<grid, CT, 0, st>>>(a);
    else if (bk32) k_conv<32, 32><<<grid, CT, 0, st>>>(a);
    else k_conv<32, 16><<<grid, CT, 0, st>>>(a);
    return cudaGetLastError();
}

int64_t wgrad_chunks(const WgradArgs &a) {
    const int64_t P = (int64_t)a.B * a.H * a.W;
    const int64_t tiles = (int64_t)(a.Cout / 32) * (a.Cin / (a.Cin % 32 == 0 ? 32 : 16)) * a.T;
    int64_t chunks = (1216 + tiles - 1) / tiles;   // about 8 blocks per SM over the GPU
    const int64_t max_chunks = (P + 255) / 256;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    return chunks;
}

cudaError_t conv_wgrad(WgradArgs a, float *dw, cudaStream_t st) {
    if (a.Cout % 32 || a.Cin % 16) return cudaErrorInvalidValue;
    const int64_t P = (int64_t)a.B * a.H * a.W;
    const int64_t chunks = wgrad_chunks(a);
    a.chunk_pixels = (P + chunks - 1) / chunks;
    a.chunk_pixels = (a.chunk_pixels + 31) / 32 * 32;
    const int64_t nchunks = (P + a.chunk_pixels - 1) / a.chunk_pixels;
    const bool c32 = a.Cin % 32 == 0;
    dim3 grid((unsigned)(a.Cout / 32), (unsigned)(a.Cin / (c32 ? 32 : 16)), (unsigned)(a.T * nchunks));
    if (c32) k_conv_wgrad<32><<<grid, 128, 0, st>>>(a);
    else k_conv_wgrad<16><<<grid, 128, 0, st>>>(a);
    const int64_t count = (int64_t)a.Cout * a.T * a.Cin;
    k_reduce_chunks<<<nb(count), 256, 0, st>>>(a.part, (int)nchunks, count, dw);
    return cudaGetLastError();
}

cudaError_t reduce_chunks(const float *part, int chunks, int64_t count, float *out, cudaStream_t st) {
    k_reduce_chunks<<<nb(count), 256, 0, st>>>(part, chunks, count, out);
    return cudaGetLastError();
}

cudaError_t bias_grad(const __nv_bfloat16 *g, int64_t P, int C, float *db, float *part, int64_t part_cap,
                      cudaStream_t st) {
    if (C < 1 || C > 256) return cudaErrorInvalidValue;
    int64_t chunks = 1216;                      // about 8 blocks per SM
    if (chunks * C > part_cap) chunks = part_cap / C;
    if (chunks > P) chunks = P;
    if (chunks < 1) return cudaErrorInvalidValue;
    const int64_t per_chunk = (P + chunks - 1) / chunks;
    chunks = (P + per_chunk - 1) / per_chunk;
    k_bias_part<<<(unsigned)chunks, 256, 0, st>>>(g, P, C, per_chunk, part);
    k_reduce_chunks_wide<<<(unsigned)C, 256, 0, st>>>(part, (int)chunks, C, db);
    return cudaGetLastError();
}

cudaError_t flip_transpose(const __nv_bfloat16 *w, int Cout, int T, int Cin, __nv_bfloat16 *wt, cudaStream_t st) {
    k_flip_transpose<<<nb((int64_t)Cout * T * Cin), 256, 0, st>>>(w, Cout, T, Cin, wt);
    return cudaGetLastError();
}

cudaError_t relu_bwd(const __nv_bfloat16 *y, const __nv_bfloat16 *dy, __nv_bfloat16 *dx, int64_t n, cudaStream_t st) {
    k_relu_bwd<<<nb(n), 256, 0, st>>>(y, dy, dx, n);
    return cudaGetLastError();
}

cudaError_t pool(const __nv_bfloat16 *x, int B, int H, int W, int C, __nv_bfloat16 *y, cudaStream_t st) {
    k_pool<<<nb((int64_t)B * (H / 2) * (W / 2) * C), 256, 0, st>>>(x, B, H, W, C, y);
    return cudaGetLastError();
}

cudaError_t pool_bwd_add(const __nv_bfloat16 *dy, int B, int H, int W, int C, __nv_bfloat16 *dx, cudaStream_t st) {
    k_pool_bwd_add<<<nb((int64_t)B * H * W * C), 256, 0, st>>>(dy, B, H, W, C, dx);
    return cudaGetLastError();
}

cudaError_t up_add(const __nv_bfloat16 *r, const __nv_bfloat16 *s, int B, int H, int W, int C, __nv_bfloat16 *y,
                   cudaStream_t st) {
    k_up_add<<<nb((int64_t)B * H * W * C), 256, 0, st>>>(r, s, B, H, W, C, y);
    return cudaGetLastError();
}

cudaError_t down_sum(const __nv_bfloat16 *dy, int B, int H, int W, int C, __nv_bfloat16 *dr, cudaStream_t st) {
    k_down_sum<<<nb((int64_t)B * (H / 2) * (W / 2) * C), 256, 0, st>>>(dy, B, H, W, C, dr);
    return cudaGetLastError();
}

cudaError_t add_into(const __nv_bfloat16 *a, __nv_bfloat16 *b, int64_t n, cudaStream_t st) {
    k_add<<<nb(n), 256, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

cudaError_t head(const __nv_bfloat16 *x, int64_t P, int C, const float *w, const float *b, float *out,
                 cudaStream_t st) {
    k_head<<<nb(P), 256, 0, st>>>(x, P, C, w, b, out);
    return cudaGetLastError();
}

cudaError_t loss(const float *out, const float *target, int64_t P, float *dout, float *part, int parts,
                 cudaStream_t st) {
    k_loss<<<parts, 256, 0, st>>>(out, target, P, dout, part);
    return cudaGetLastError();
}

cudaError_t head_bwd(const float *dout, const __nv_bfloat16 *x, int64_t P, int C, const float *w,
                     __nv_bfloat16 *dx, float *part, float *dwb, cudaStream_t st) {
    k_head_bwd_x<<<nb(P * C), 256, 0, st>>>(dout, P, C, w, dx);
    const int blocks = (int)((P + 1023) / 1024);
    const int K = 2 * C + 2;
    k_head_bwd_w<<<blocks, 128, sizeof(float) * K, st>>>(dout, x, P, C, part);
    k_reduce_chunks<<<nb(K), 256, 0, st>>>(part, blocks, K, dwb);
    return cudaGetLastError();
}

cudaError_t adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                 int step, __nv_bfloat16 *w16, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<nb(n), 256, 0, st>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2, w16);
    return cudaGetLastError();
}

cudaError_t to_bf16(const float *x, __nv_bfloat16 *y, int64_t n, cudaStream_t st) {
    k_to_bf16<<<nb(n), 256, 0, st>>>(x, y, n);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace gabp
