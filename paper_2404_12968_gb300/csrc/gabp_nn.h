// Internal interface of the warm-start network kernels (gabp_nn_kernels.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gabp {
namespace nn {

// out = act(conv(in, w) + bias (+ skip)); NHWC BF16, weights [Cout][T][Cin], T = 9 or 1.
// Cout a multiple of 32, Cin a multiple of 16.
struct ConvArgs {
    const __nv_bfloat16 *in;
    const __nv_bfloat16 *w;
    const float *bias;          // may be NULL
    const __nv_bfloat16 *skip;  // may be NULL; [B][H][W][Cout]
    __nv_bfloat16 *out;
    int B, H, W, Cin, Cout, T, relu;
};

// dw[co][t][ci] = sum_p g[p][co] in[p + d_t][ci]; `part` holds chunk partials
// (wgrad_chunks(args) * Cout * T * Cin floats).
struct WgradArgs {
    const __nv_bfloat16 *g;     // [B][H][W][Cout]
    const __nv_bfloat16 *in;    // [B][H][W][Cin]
    float *part;
    int B, H, W, Cin, Cout, T;
    int64_t chunk_pixels;       // set by conv_wgrad
};

cudaError_t conv(const ConvArgs &a, cudaStream_t st);

// Forward convolution on the tcgen05 tensor cores (gabp_nn_tc.cu): out = act(conv(in, w) + bias)
// with optional fused 2x2 average pooling, nearest upsampling plus skip, and 1x1 FP32 head.
// Input [B][H][W][Cin] BF16 (given separately, read through a TMA tensor map); Cin a multiple
// of 16, Cout 32, 64, 128 or 256; H and W even when pooling.  The weights are prepacked by
// tc_pack_weights.
struct TcConvArgs {
    const __nv_bfloat16 *wpk;     // packed weights (tc_pack_weights)
    const float *bias;            // [Cout]
    __nv_bfloat16 *out;           // [B][H][W][Cout], or NULL
    __nv_bfloat16 *pool_out;      // 2x2 average of out, [B][H/2][W/2][Cout], or NULL
    const __nv_bfloat16 *up_skip; // [B][2H][2W][Cout] (with up_out)
    __nv_bfloat16 *up_out;        // nearest-upsampled out + up_skip, [B][2H][2W][Cout], or NULL
    const float *head_w;          // [2][Cout] FP32 head (Cout = 32), or NULL
    const float *head_b;          // [2]
    float *head_out;              // [B][H][W][2] FP32
    int *err;                     // device flag, set if a bounded wait ran out
    int B, H, W, Cin, Cout, T, relu;
    // set by tc_conv
    int stages, nblocks, tiles_x, tiles_y, resident;
    int64_t ntiles;
};
int tc_block_n(int Cout);
// packed[nb][kb][t][h][n][e] = w[nb * N + n][t][16 kb + 8 h + e], N = tc_block_n(Cout)
cudaError_t tc_pack_weights(const __nv_bfloat16 *w, int Cout, int T, int Cin, __nv_bfloat16 *out, cudaStream_t st);
cudaError_t tc_conv(const __nv_bfloat16 *in, TcConvArgs a, cudaStream_t st);
int64_t wgrad_chunks(const WgradArgs &a);
cudaError_t conv_wgrad(WgradArgs a, float *dw, cudaStream_t st);
// Weight gradient on the tcgen05 tensor cores (gabp_nn_tc.cu): dw[co][t][ci] = sum over the
// pixels p of g[p][co] in[p + d_t][ci] (zero outside the image), as partial sums over pixel
// chunks in part (at most part_cap floats) reduced into dw in chunk order.  Cin a multiple
// of 16 (at most 256 per block of N), any Cout (blocks of 128; rows past Cout are zero).
struct TcWgradArgs {
    const __nv_bfloat16 *g;     // [B][H][W][Cout]
    const __nv_bfloat16 *in;    // [B][H][W][Cin]
    float *part;
    int64_t part_cap;
    int *err;                   // device flag, set if a bounded wait ran out
    int B, H, W, Cin, Cout, T;
    // set by tc_wgrad
    int N, nbn, nbm, chunks, stages, ky, ga, tpc, ngroups;
    int64_t ktiles, tiles_x, tiles_y, per_chunk;
};
cudaError_t tc_wgrad(TcWgradArgs a, float *dw, cudaStream_t st);
// out[i] = sum over c < chunks of part[c * count + i], in chunk order
cudaError_t reduce_chunks(const float *part, int chunks, int64_t count, float *out, cudaStream_t st);
// db[c] = sum over the P pixels of g[p][c]: chunk partials in part (at most part_cap floats),
// reduced in chunk order; C at most 256
cudaError_t bias_grad(const __nv_bfloat16 *g, int64_t P, int C, float *db, float *part, int64_t part_cap,
                      cudaStream_t st);
cudaError_t flip_transpose(const __nv_bfloat16 *w, int Cout, int T, int Cin, __nv_bfloat16 *wt, cudaStream_t st);
cudaError_t relu_bwd(const __nv_bfloat16 *y, const __nv_bfloat16 *dy, __nv_bfloat16 *dx, int64_t n, cudaStream_t st);
cudaError_t pool(const __nv_bfloat16 *x, int B, int H, int W, int C, __nv_bfloat16 *y, cudaStream_t st);
cudaError_t pool_bwd_add(const __nv_bfloat16 *dy, int B, int H, int W, int C, __nv_bfloat16 *dx, cudaStream_t st);
cudaError_t up_add(const __nv_bfloat16 *r, const __nv_bfloat16 *s, int B, int H, int W, int C, __nv_bfloat16 *y,
                   cudaStream_t st);
cudaError_t down_sum(const __nv_bfloat16 *dy, int B, int H, int W, int C, __nv_bfloat16 *dr, cudaStream_t st);
cudaError_t add_into(const __nv_bfloat16 *a, __nv_bfloat16 *b, int64_t n, cudaStream_t st);
cudaError_t head(const __nv_bfloat16 *x, int64_t P, int C, const float *w, const float *b, float *out,
                 cudaStream_t st);
cudaError_t loss(const float *out, const float *target, int64_t P, float *dout, float *part, int parts,
                 cudaStream_t st);
// dx (BF16) and the head's weight/bias gradients dwb[2C + 2] (part: ceil(P/1024) * (2C+2) floats)
cudaError_t head_bwd(const float *dout, const __nv_bfloat16 *x, int64_t P, int C, const float *w,
                     __nv_bfloat16 *dx, float *part, float *dwb, cudaStream_t st);
cudaError_t adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                 int step, __nv_bfloat16 *w16, cudaStream_t st);
cudaError_t to_bf16(const float *x, __nv_bfloat16 *y, int64_t n, cudaStream_t st);

}  // namespace nn
}  // namespace gabp
