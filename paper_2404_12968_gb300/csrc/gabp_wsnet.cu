// The learned warm start's network: a 4-level convolutional encoder-decoder (32, 64, 128,
// 256 channels) mapping [observed value, observation mask, log kappa] on the grid to initial
// beliefs [mean / scale, log precision].  BF16 weights and activations, FP32 accumulation and
// FP32 master weights (Adam).  Forward and backward run on the kernels of gabp_nn_kernels.cu.
//
// Layers (NHWC, 3x3 convolutions with zero padding unless noted):
//   enc0: 16->32, 32->32 (s0)  | pool | enc1: 32->64, 64->64 (s1) | pool |
//   enc2: 64->128, 128->128 (s2) | pool | enc3: 128->256, 256->256 (b3)
//   dec2: r2 = 1x1 256->128 at 1/8, u2 = up(r2) + s2, d2 = 128->128
//   dec1: r1 = 1x1 128->64, u1 = up(r1) + s1, d1 = 64->64
//   dec0: r0 = 1x1 64->32,  u0 = up(r0) + s0, d0 = 32->32
//   head: 1x1 32->2, FP32 out.   ReLU after every 3x3 convolution; none after the 1x1 ones.
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "gabp.h"
#include "gabp_internal.h"
#include "gabp_nn.h"

using gabp::nn::ConvArgs;
using gabp::nn::WgradArgs;

namespace {

struct LayerSpec {
    int cin, cout, taps, relu;
};

constexpr int NLAYER = 14;
constexpr LayerSpec SPECS[NLAYER] = {
    {16, 32, 9, 1},  {32, 32, 9, 1},   {32, 64, 9, 1},   {64, 64, 9, 1},   {64, 128, 9, 1},
    {128, 128, 9, 1}, {128, 256, 9, 1}, {256, 256, 9, 1}, {256, 128, 1, 0}, {128, 128, 9, 1},
    {128, 64, 1, 0},  {64, 64, 9, 1},   {64, 32, 1, 0},   {32, 32, 9, 1}};
constexpr int HEAD_C = 32;

struct Buf {
    __nv_bfloat16 *p = nullptr;
    int64_t n = 0;
};

}  // namespace

struct gabp_wsnet {
    int dev = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t woff[NLAYER + 1] = {0};   // offsets of each layer's weights in the flat vector
    int64_t boff[NLAYER] = {0};       // offsets of each layer's bias
    int64_t head_off = 0, nparam = 0; // head: w[2][32] then b[2]
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // FP32 master, Adam, grads
    __nv_bfloat16 *w16 = nullptr;    // BF16 copy (the flat vector, converted)
    __nv_bfloat16 *wt = nullptr;     // flipped/transposed weights scratch (largest layer)
    __nv_bfloat16 *wpk = nullptr;    // weights packed for the tensor-core forward (same offsets)
    __nv_bfloat16 *wtpk = nullptr;   // flipped/transposed weights packed for the tensor-core backward (largest layer)
    float *zbias = nullptr;          // 256 zeros: the backward-data convolution has no bias
    bool packed = false;             // wpk matches w16
    int *derr = nullptr;             // device flag of the tensor-core kernels (a bounded wait ran out)
    int kernels = GABP_WSNET_TCGEN05;
    const __nv_bfloat16 *xin = nullptr;   // caller's input, read in place by the tensor-core forward
    int step = 0;
    // activation buffers for the current shape
    int B = 0, H = 0, W = 0;
    bool grads = false;
    Buf x, a0, s0, p0, a1, s1, p1, a2, s2, p2, a3, b3, r2, u2, d2, r1, u1, d1, r0, u0, d0;
    Buf ga, gb, gs0, gs1, gs2, gr;   // gradient scratch
    float *out = nullptr, *dout = nullptr, *part = nullptr;
    int64_t part_n = 0;
    std::vector<void *> act_allocs;
};

namespace {

thread_local std::string t_ws_err;

int wfail(gabp_wsnet *n, int code, const std::string &msg) {
    if (n) n->err = msg;
    else t_ws_err = msg;
    return code;
}

int wcuda(gabp_wsnet *n, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    return wfail(n, e == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA, m);
}

#define WK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return wcuda(net, e_, what); \
    } while (0)

void free_acts(gabp_wsnet *net) {
    for (void *q : net->act_allocs) cudaFree(q);
    net->act_allocs.clear();
    net->B = net->H = net->W = 0;
    net->grads = false;
}

int alloc_buf(gabp_wsnet *net, Buf &b, int64_t n) {
    b.n = n;
    void *q = nullptr;
    WK(cudaMalloc(&q, sizeof(__nv_bfloat16) * (n > 0 ? n : 1)), "alloc activation");
    net->act_allocs.push_back(q);
    b.p = (__nv_bfloat16 *)q;
    return GABP_OK;
}

int ensure_shape(gabp_wsnet *net, int B, int H, int W, bool grads) {
    if (net->B == B && net->H == H && net->W == W && (net->grads || !grads)) return GABP_OK;
    free_acts(net);
    const int64_t P0 = (int64_t)B * H * W, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
    int rc = 0;
    struct {
        Buf *b;
        int64_t n;
    } L[] = {{&net->x, P0 * 16},  {&net->a0, P0 * 32}, {&net->s0, P0 * 32}, {&net->p0, P1 * 32},
             {&net->a1, P1 * 64}, {&net->s1, P1 * 64}, {&net->p1, P2 * 64}, {&net->a2, P2 * 128},
             {&net->s2, P2 * 128}, {&net->p2, P3 * 128}, {&net->a3, P3 * 256}, {&net->b3, P3 * 256},
             {&net->r2, P3 * 128}, {&net->u2, P2 * 128}, {&net->d2, P2 * 128}, {&net->r1, P2 * 64},
             {&net->u1, P1 * 64}, {&net->d1, P1 * 64},  {&net->r0, P1 * 32}, {&net->u0, P0 * 32},
             {&net->d0, P0 * 32}};
    for (auto &e : L)
        if ((rc = alloc_buf(net, *e.b, e.n))) return rc;
    void *q = nullptr;
    WK(cudaMalloc(&q, sizeof(float) * 2 * P0), "alloc output");
    net->act_allocs.push_back(q);
    net->out = (float *)q;
    if (grads) {
        // gradient scratch: two ping-pong buffers of the largest activation, one per skip level,
        // one for the 1x1 reductions
        const int64_t big = P0 * 32 > P1 * 64 ? P0 * 32 : P1 * 64;
        if ((rc = alloc_buf(net, net->ga, big))) return rc;
        if ((rc = alloc_buf(net, net->gb, big))) return rc;
        if ((rc = alloc_buf(net, net->gs0, P0 * 32))) return rc;
        if ((rc = alloc_buf(net, net->gs1, P1 * 64))) return rc;
        if ((rc = alloc_buf(net, net->gs2, P2 * 128))) return rc;
        if ((rc = alloc_buf(net, net->gr, P1 * 64 > P0 * 16 ? P1 * 64 : P0 * 16))) return rc;
        WK(cudaMalloc(&q, sizeof(float) * 2 * P0), "alloc output grad");
        net->act_allocs.push_back(q);
        net->dout = (float *)q;
        // partial sums of the weight gradients (largest layer), the head and the loss
        int64_t need = 0;
        const int Hs[NLAYER] = {H, H, H / 2, H / 2, H / 4, H / 4, H / 8, H / 8, H / 8, H / 4, H / 4, H / 2, H / 2, H};
        for (int l = 0; l < NLAYER; ++l) {
            WgradArgs wa{};
            wa.B = B;
            wa.H = Hs[l];
            wa.W = Hs[l] * W / H;
            wa.Cin = SPECS[l].cin;
            wa.Cout = SPECS[l].cout;
            wa.T = SPECS[l].taps;
            const int64_t count = (int64_t)SPECS[l].cout * SPECS[l].taps * SPECS[l].cin;
            const int64_t c = gabp::nn::wgrad_chunks(wa) * count;
            need = c > need ? c : need;
            // the tensor-core weight gradient: up to 32 pixel chunks of partial sums per layer
            // (enough blocks for the wide, shallow layers: 256 x 256 x 9 over 64^2 pixels)
            const int64_t c32 = 32 * count;
            need = c32 > need ? c32 : need;
        }
        const int64_t hp = ((P0 + 1023) / 1024) * (2 * HEAD_C + 2);
        need = need > hp ? need : hp;
        need = need > 4096 ? need : 4096;
        WK(cudaMalloc(&q, sizeof(float) * need), "alloc partials");
        net->act_allocs.push_back(q);
        net->part = (float *)q;
        net->part_n = need;
    }
    net->B = B;
    net->H = H;
    net->W = W;
    net->grads = grads;
    return GABP_OK;
}

int conv_fwd(gabp_wsnet *net, int l, const Buf &in, const Buf *skip, Buf &out, int B, int H, int W) {
    ConvArgs a{};
    a.in = in.p;
    a.w = net->w16 + net->woff[l];
    a.bias = net->w + net->boff[l];
    a.skip = skip ? skip->p : nullptr;
    a.out = out.p;
    a.B = B;
    a.H = H;
    a.W = W;
    a.Cin = SPECS[l].cin;
    a.Cout = SPECS[l].cout;
    a.T = SPECS[l].taps;
    a.relu = SPECS[l].relu;
    WK(gabp::nn::conv(a, net->stream), "conv forward");
    return GABP_OK;
}

// Forward on the tcgen05 tensor-core convolutions, with the pooling, the upsampling additions
// and the head fused into the convolutions' epilogues.  Buffers that only the backward pass
// reads (r2, r1, r0, d0) are written when gradients are wanted.
int forward_tc(gabp_wsnet *net) {
    const int B = net->B, H = net->H, W = net->W;
    cudaStream_t st = net->stream;
    if (!net->packed) {
        for (int l = 0; l < NLAYER; ++l)
            WK(gabp::nn::tc_pack_weights(net->w16 + net->woff[l], SPECS[l].cout, SPECS[l].taps, SPECS[l].cin,
                                         net->wpk + net->woff[l], st),
               "pack weights");
        net->packed = true;
    }
    const bool keep = net->grads;
    auto L = [&](int l, const Buf &in, int h, int w, Buf *out, Buf *pool, const Buf *up_skip, Buf *up,
                 bool head) -> int {
        gabp::nn::TcConvArgs a{};
        a.wpk = net->wpk + net->woff[l];
        a.bias = net->w + net->boff[l];
        a.out = out ? out->p : nullptr;
        a.pool_out = pool ? pool->p : nullptr;
        a.up_skip = up_skip ? up_skip->p : nullptr;
        a.up_out = up ? up->p : nullptr;
        if (head) {
            a.head_w = net->w + net->head_off;
            a.head_b = net->w + net->head_off + 2 * HEAD_C;
            a.head_out = net->out;
        }
        a.err = net->derr;
        a.B = B;
        a.H = h;
        a.W = w;
        a.Cin = SPECS[l].cin;
        a.Cout = SPECS[l].cout;
        a.T = SPECS[l].taps;
        a.relu = SPECS[l].relu;
        WK(gabp::nn::tc_conv(in.p, a, st), "tensor-core convolution");
        return GABP_OK;
    };
    int rc;
#define F(...) \
    if ((rc = L(__VA_ARGS__))) return rc
    Buf xin;
    xin.p = const_cast<__nv_bfloat16 *>(net->xin ? net->xin : net->x.p);
    xin.n = net->x.n;
    F(0, xin, H, W, &net->a0, nullptr, nullptr, nullptr, false);
    F(1, net->a0, H, W, &net->s0, &net->p0, nullptr, nullptr, false);
    F(2, net->p0, H / 2, W / 2, &net->a1, nullptr, nullptr, nullptr, false);
    F(3, net->a1, H / 2, W / 2, &net->s1, &net->p1, nullptr, nullptr, false);
    F(4, net->p1, H / 4, W / 4, &net->a2, nullptr, nullptr, nullptr, false);
    F(5, net->a2, H / 4, W / 4, &net->s2, &net->p2, nullptr, nullptr, false);
    F(6, net->p2, H / 8, W / 8, &net->a3, nullptr, nullptr, nullptr, false);
    F(7, net->a3, H / 8, W / 8, &net->b3, nullptr, nullptr, nullptr, false);
    F(8, net->b3, H / 8, W / 8, keep ? &net->r2 : nullptr, nullptr, &net->s2, &net->u2, false);
    F(9, net->u2, H / 4, W / 4, &net->d2, nullptr, nullptr, nullptr, false);
    F(10, net->d2, H / 4, W / 4, keep ? &net->r1 : nullptr, nullptr, &net->s1, &net->u1, false);
    F(11, net->u1, H / 2, W / 2, &net->d1, nullptr, nullptr, nullptr, false);
    F(12, net->d1, H / 2, W / 2, keep ? &net->r0 : nullptr, nullptr, &net->s0, &net->u0, false);
    F(13, net->u0, H, W, keep ? &net->d0 : nullptr, nullptr, nullptr, nullptr, true);
#undef F
    return GABP_OK;
}

int forward(gabp_wsnet *net) {
    if (net->kernels == GABP_WSNET_TCGEN05) return forward_tc(net);
    const int B = net->B, H = net->H, W = net->W;
    cudaStream_t st = net->stream;
    int rc;
#define F(l, in, skip, out, h, w) \
    if ((rc = conv_fwd(net, l, in, skip, out, B, h, w))) return rc
    F(0, net->x, nullptr, net->a0, H, W);
    F(1, net->a0, nullptr, net->s0, H, W);
    WK(gabp::nn::pool(net->s0.p, B, H, W, 32, net->p0.p, st), "pool");
    F(2, net->p0, nullptr, net->a1, H / 2, W / 2);
    F(3, net->a1, nullptr, net->s1, H / 2, W / 2);
    WK(gabp::nn::pool(net->s1.p, B, H / 2, W / 2, 64, net->p1.p, st), "pool");
    F(4, net->p1, nullptr, net->a2, H / 4, W / 4);
    F(5, net->a2, nullptr, net->s2, H / 4, W / 4);
    WK(gabp::nn::pool(net->s2.p, B, H / 4, W / 4, 128, net->p2.p, st), "pool");
    F(6, net->p2, nullptr, net->a3, H / 8, W / 8);
    F(7, net->a3, nullptr, net->b3, H / 8, W / 8);
    F(8, net->b3, nullptr, net->r2, H / 8, W / 8);
    WK(gabp::nn::up_add(net->r2.p, net->s2.p, B, H / 4, W / 4, 128, net->u2.p, st), "up");
    F(9, net->u2, nullptr, net->d2, H / 4, W / 4);
    F(10, net->d2, nullptr, net->r1, H / 4, W / 4);
    WK(gabp::nn::up_add(net->r1.p, net->s1.p, B, H / 2, W / 2, 64, net->u1.p, st), "up");
    F(11, net->u1, nullptr, net->d1, H / 2, W / 2);
    F(12, net->d1, nullptr, net->r0, H / 2, W / 2);
    WK(gabp::nn::up_add(net->r0.p, net->s0.p, B, H, W, 32, net->u0.p, st), "up");
    F(13, net->u0, nullptr, net->d0, H, W);
#undef F
    WK(gabp::nn::head(net->d0.p, (int64_t)B * H * W, HEAD_C, net->w + net->head_off, net->w + net->head_off + 2 * HEAD_C,
                      net->out, st),
       "head");
    return GABP_OK;
}

// gradient of layer l given the gradient g (after the activation's backward) at its output;
// writes dW, db into net->g and, if din, the gradient w.r.t. its input
int conv_bwd(gabp_wsnet *net, int l, const Buf &g, const Buf &in, Buf *din, int h, int w) {
    const int B = net->B;
    cudaStream_t st = net->stream;
    const LayerSpec &s = SPECS[l];
    WgradArgs wa{};
    wa.g = g.p;
    wa.in = in.p;
    wa.part = net->part;
    wa.B = B;
    wa.H = h;
    wa.W = w;
    wa.Cin = s.cin;
    wa.Cout = s.cout;
    wa.T = s.taps;
    if (net->kernels == GABP_WSNET_TCGEN05) {
        gabp::nn::TcWgradArgs ta{};
        ta.g = g.p;
        ta.in = in.p;
        ta.part = net->part;
        ta.part_cap = net->part_n;
        ta.err = net->derr;
        ta.B = B;
        ta.H = h;
        ta.W = w;
        ta.Cin = s.cin;
        ta.Cout = s.cout;
        ta.T = s.taps;
        WK(gabp::nn::tc_wgrad(ta, net->g + net->woff[l], st), "tensor-core weight gradient");
    } else {
        WK(gabp::nn::conv_wgrad(wa, net->g + net->woff[l], st), "conv wgrad");
    }
    WK(gabp::nn::bias_grad(g.p, (int64_t)B * h * w, s.cout, net->g + net->boff[l], net->part, net->part_n, st),
       "bias grad");
    if (din && net->kernels == GABP_WSNET_TCGEN05) {
        // gradient w.r.t. the input: the forward convolution of g with the flipped, transposed
        // weights (Cin and Cout exchanged), on the tcgen05 tensor cores like the forward pass
        WK(gabp::nn::flip_transpose(net->w16 + net->woff[l], s.cout, s.taps, s.cin, net->wt, st), "flip");
        WK(gabp::nn::tc_pack_weights(net->wt, s.cin, s.taps, s.cout, net->wtpk, st), "pack flipped weights");
        gabp::nn::TcConvArgs a{};
        a.wpk = net->wtpk;
        a.bias = net->zbias;
        a.out = din->p;
        a.err = net->derr;
        a.B = B;
        a.H = h;
        a.W = w;
        a.Cin = s.cout;
        a.Cout = s.cin;
        a.T = s.taps;
        a.relu = 0;
        WK(gabp::nn::tc_conv(g.p, a, st), "tensor-core convolution backward data");
    } else if (din) {
        WK(gabp::nn::flip_transpose(net->w16 + net->woff[l], s.cout, s.taps, s.cin, net->wt, st), "flip");
        ConvArgs a{};
        a.in = g.p;
        a.w = net->wt;
        a.out = din->p;
        a.B = B;
        a.H = h;
        a.W = w;
        a.Cin = s.cout;
        a.Cout = s.cin;
        a.T = s.taps;
        WK(gabp::nn::conv(a, st), "conv backward data");
    }
    return GABP_OK;
}

int backward(gabp_wsnet *net) {
    const int B = net->B, H = net->H, W = net->W;
    const int64_t P0 = (int64_t)B * H * W;
    cudaStream_t st = net->stream;
    int rc;
    Buf &ga = net->ga, &gb = net->gb;
    // head
    WK(gabp::nn::head_bwd(net->dout, net->d0.p, P0, HEAD_C, net->w + net->head_off, ga.p, net->part,
                          net->g + net->head_off, st),
       "head backward");
    // dec0
    WK(gabp::nn::relu_bwd(net->d0.p, ga.p, gb.p, P0 * 32, st), "relu bwd");
    if ((rc = conv_bwd(net, 13, gb, net->u0, &net->gs0, H, W))) return rc;        // gs0 = du0
    WK(gabp::nn::down_sum(net->gs0.p, B, H, W, 32, net->gr.p, st), "down");        // gr = dr0
    if ((rc = conv_bwd(net, 12, net->gr, net->d1, &ga, H / 2, W / 2))) return rc;  // ga = dd1
    // dec1
    WK(gabp::nn::relu_bwd(net->d1.p, ga.p, gb.p, P0 / 4 * 64, st), "relu bwd");
    if ((rc = conv_bwd(net, 11, gb, net->u1, &net->gs1, H / 2, W / 2))) return rc;  // gs1 = du1
    WK(gabp::nn::down_sum(net->gs1.p, B, H / 2, W / 2, 64, net->gr.p, st), "down"); // gr = dr1
    if ((rc = conv_bwd(net, 10, net->gr, net->d2, &ga, H / 4, W / 4))) return rc;   // ga = dd2
    // dec2
    WK(gabp::nn::relu_bwd(net->d2.p, ga.p, gb.p, P0 / 16 * 128, st), "relu bwd");
    if ((rc = conv_bwd(net, 9, gb, net->u2, &net->gs2, H / 4, W / 4))) return rc;   // gs2 = du2
    WK(gabp::nn::down_sum(net->gs2.p, B, H / 4, W / 4, 128, net->gr.p, st), "down"); // gr = dr2
    if ((rc = conv_bwd(net, 8, net->gr, net->b3, &ga, H / 8, W / 8))) return rc;     // ga = db3
    // enc3
    WK(gabp::nn::relu_bwd(net->b3.p, ga.p, gb.p, P0 / 64 * 256, st), "relu bwd");
    if ((rc = conv_bwd(net, 7, gb, net->a3, &ga, H / 8, W / 8))) return rc;          // ga = da3
    WK(gabp::nn::relu_bwd(net->a3.p, ga.p, gb.p, P0 / 64 * 256, st), "relu bwd");
    if ((rc = conv_bwd(net, 6, gb, net->p2, &ga, H / 8, W / 8))) return rc;          // ga = dp2
    WK(gabp::nn::pool_bwd_add(ga.p, B, H / 4, W / 4, 128, net->gs2.p, st), "pool bwd");
    // enc2
    WK(gabp::nn::relu_bwd(net->s2.p, net->gs2.p, gb.p, P0 / 16 * 128, st), "relu bwd");
    if ((rc = conv_bwd(net, 5, gb, net->a2, &ga, H / 4, W / 4))) return rc;          // ga = da2
    WK(gabp::nn::relu_bwd(net->a2.p, ga.p, gb.p, P0 / 16 * 128, st), "relu bwd");
    if ((rc = conv_bwd(net, 4, gb, net->p1, &ga, H / 4, W / 4))) return rc;          // ga = dp1
    WK(gabp::nn::pool_bwd_add(ga.p, B, H / 2, W / 2, 64, net->gs1.p, st), "pool bwd");
    // enc1
    WK(gabp::nn::relu_bwd(net->s1.p, net->gs1.p, gb.p, P0 / 4 * 64, st), "relu bwd");
    if ((rc = conv_bwd(net, 3, gb, net->a1, &ga, H / 2, W / 2))) return rc;          // ga = da1
    WK(gabp::nn::relu_bwd(net->a1.p, ga.p, gb.p, P0 / 4 * 64, st), "relu bwd");
    if ((rc = conv_bwd(net, 2, gb, net->p0, &ga, H / 2, W / 2))) return rc;          // ga = dp0
    WK(gabp::nn::pool_bwd_add(ga.p, B, H, W, 32, net->gs0.p, st), "pool bwd");
    // enc0
    WK(gabp::nn::relu_bwd(net->s0.p, net->gs0.p, gb.p, P0 * 32, st), "relu bwd");
    if ((rc = conv_bwd(net, 1, gb, net->a0, &ga, H, W))) return rc;                  // ga = da0
    WK(gabp::nn::relu_bwd(net->a0.p, ga.p, gb.p, P0 * 32, st), "relu bwd");
    if ((rc = conv_bwd(net, 0, gb, net->x, nullptr, H, W))) return rc;
    return GABP_OK;
}

int check_shape(gabp_wsnet *net, int B, int H, int W) {
    if (B < 1 || H < 8 || W < 8 || H % 8 || W % 8) return wfail(net, GABP_ERR_ARG, "B >= 1 and H, W multiples of 8 (>= 8)");
    return GABP_OK;
}

}  // namespace

namespace gabp {

// forward on a device input [1][H][W][16] already in the net's input buffer layout
int wsnet_forward_device(gabp_wsnet *net, const void *x, int B, int H, int W, float **out, cudaStream_t st,
                         std::string &err) {
    int rc = check_shape(net, B, H, W);
    if (!rc) rc = ensure_shape(net, B, H, W, false);
    if (rc) {
        err = net->err;
        return rc;
    }
    cudaStream_t keep = net->stream;
    net->stream = st;
    if (net->kernels == GABP_WSNET_TCGEN05) {
        net->xin = (const __nv_bfloat16 *)x;   // the first convolution reads the input in place
    } else {
        cudaError_t e = cudaMemcpyAsync(net->x.p, x, sizeof(__nv_bfloat16) * net->x.n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            net->stream = keep;
            err = cudaGetErrorString(e);
            return GABP_ERR_CUDA;
        }
    }
    rc = forward(net);
    net->xin = nullptr;
    net->stream = keep;
    if (rc) err = net->err;
    *out = net->out;
    return rc;
}

int wsnet_device(const gabp_wsnet *net) { return net->dev; }

// After a synchronisation: 1 if a tensor-core kernel's bounded wait ran out (flag cleared).
int wsnet_take_device_error(gabp_wsnet *net) {
    int h = 0;
    if (cudaMemcpy(&h, net->derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    if (h) cudaMemset(net->derr, 0, sizeof(int));
    return h ? 1 : 0;
}

}  // namespace gabp

extern "C" {

const char *gabp_wsnet_create_error(void) { return t_ws_err.c_str(); }

int gabp_wsnet_create(gabp_wsnet **out, uint64_t seed, int device) {
    t_ws_err.clear();
    if (!out) return wfail(nullptr, GABP_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    gabp_wsnet *net = new (std::nothrow) gabp_wsnet();
    if (!net) return GABP_ERR_OOM;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete net;
        return wfail(nullptr, GABP_ERR_CUDA, "no CUDA device");
    }
    net->dev = dev;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    int64_t off = 0;
    for (int l = 0; l < NLAYER; ++l) {
        net->woff[l] = off;
        off += (int64_t)SPECS[l].cout * SPECS[l].taps * SPECS[l].cin;
        net->boff[l] = off;
        off += SPECS[l].cout;
    }
    net->head_off = off;
    off += 2 * HEAD_C + 2;
    net->nparam = off;
    // He-normal initialisation (seeded), zero biases; the head starts small
    std::vector<float> h(off, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int l = 0; l < NLAYER; ++l) {
        const int64_t fan_in = (int64_t)SPECS[l].taps * (l == 0 ? 3 : SPECS[l].cin);
        const float sd = std::sqrt(2.f / (float)fan_in);
        for (int64_t i = net->woff[l]; i < net->boff[l]; ++i) {
            const int ci = (int)((i - net->woff[l]) % SPECS[l].cin);
            h[i] = (l == 0 && ci >= 3) ? 0.f : sd * nd(rng);   // layer 0 uses 3 of its 16 input channels
        }
    }
    for (int i = 0; i < 2 * HEAD_C; ++i) h[net->head_off + i] = 0.05f * nd(rng);
    int rc = GABP_OK;
    size_t maxw = 0;
    for (int l = 0; l < NLAYER; ++l) {
        const size_t s = (size_t)SPECS[l].cout * SPECS[l].taps * SPECS[l].cin;
        maxw = s > maxw ? s : maxw;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->w, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->m, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->v, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->g, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->w16, sizeof(__nv_bfloat16) * off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->wt, sizeof(__nv_bfloat16) * maxw);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->wpk, sizeof(__nv_bfloat16) * off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->wtpk, sizeof(__nv_bfloat16) * maxw);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->zbias, sizeof(float) * 256);
    if (e == cudaSuccess) e = cudaMemset(net->zbias, 0, sizeof(float) * 256);
    if (e == cudaSuccess) e = cudaMalloc((void **)&net->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(net->derr, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(net->w, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(net->m, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(net->v, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = gabp::nn::to_bf16(net->w, net->w16, off, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) rc = wcuda(nullptr, e, "network allocation");
    if (prev >= 0) cudaSetDevice(prev);
    if (rc) {
        gabp_wsnet_destroy(net);
        return rc;
    }
    *out = net;
    return GABP_OK;
}

int64_t gabp_wsnet_param_count(const gabp_wsnet *net) { return net ? net->nparam : -1; }

int gabp_wsnet_get_params(gabp_wsnet *net, float *params) {
    if (!net || !params) return GABP_ERR_ARG;
    WK(cudaMemcpy(params, net->w, sizeof(float) * net->nparam, cudaMemcpyDefault), "copy params");
    return GABP_OK;
}

int gabp_wsnet_set_params(gabp_wsnet *net, const float *params) {
    if (!net || !params) return GABP_ERR_ARG;
    WK(cudaMemcpy(net->w, params, sizeof(float) * net->nparam, cudaMemcpyDefault), "copy params");
    WK(gabp::nn::to_bf16(net->w, net->w16, net->nparam, net->stream), "to bf16");
    net->packed = false;
    WK(cudaStreamSynchronize(net->stream), "sync");
    return GABP_OK;
}

int gabp_wsnet_set_kernels(gabp_wsnet *net, int kernels) {
    if (!net || (kernels != GABP_WSNET_TCGEN05 && kernels != GABP_WSNET_MMA_SYNC)) return GABP_ERR_ARG;
    net->kernels = kernels;
    return GABP_OK;
}

int gabp_wsnet_forward(gabp_wsnet *net, const void *x, int B, int H, int W, float *out) {
    if (!net || !x || !out) return GABP_ERR_ARG;
    int rc = check_shape(net, B, H, W);
    if (rc) return rc;
    if ((rc = ensure_shape(net, B, H, W, net->grads))) return rc;
    WK(cudaMemcpyAsync(net->x.p, x, sizeof(__nv_bfloat16) * net->x.n, cudaMemcpyDefault, net->stream), "copy input");
    if ((rc = forward(net))) return rc;
    WK(cudaMemcpyAsync(out, net->out, sizeof(float) * 2 * B * H * W, cudaMemcpyDefault, net->stream), "copy output");
    WK(cudaStreamSynchronize(net->stream), "sync");
    if (gabp::wsnet_take_device_error(net)) return wfail(net, GABP_ERR_TIMEOUT, "a tensor-core kernel wait ran out");
    return GABP_OK;
}

// Gradients of the loss w.r.t. every parameter (flat FP32, into `grads` if not NULL) without
// updating; returns the loss.  xs / ts: B device pointers to [H][W][16] BF16 inputs and
// [H][W][2] FP32 targets.
static int grad_impl(gabp_wsnet *net, const void *const *xs, const float *const *ts, int B, int H, int W,
                     float *loss_out) {
    int rc = check_shape(net, B, H, W);
    if (rc) return rc;
    if ((rc = ensure_shape(net, B, H, W, true))) return rc;
    const int64_t per = (int64_t)H * W;
    for (int b = 0; b < B; ++b)
        WK(cudaMemcpyAsync(net->x.p + b * per * 16, xs[b], sizeof(__nv_bfloat16) * per * 16, cudaMemcpyDefault,
                           net->stream),
           "gather inputs");
    if ((rc = forward(net))) return rc;
    // the targets are staged in the dout buffer; the loss kernel replaces each target pair by
    // d loss / d out in place (each thread reads its pair before writing it)
    for (int b = 0; b < B; ++b)
        WK(cudaMemcpyAsync(net->dout + b * per * 2, ts[b], sizeof(float) * per * 2, cudaMemcpyDefault, net->stream),
           "gather targets");
    const int parts = 1024;
    WK(gabp::nn::loss(net->out, net->dout, (int64_t)B * per, net->dout, net->part, parts, net->stream), "loss");
    std::vector<float> hp(parts);
    WK(cudaMemcpyAsync(hp.data(), net->part, sizeof(float) * parts, cudaMemcpyDeviceToHost, net->stream), "copy loss");
    if ((rc = backward(net))) return rc;
    WK(cudaStreamSynchronize(net->stream), "sync");
    double l = 0.0;
    for (float v : hp) l += v;
    if (loss_out) *loss_out = (float)l;
    return GABP_OK;
}

int gabp_wsnet_gradients(gabp_wsnet *net, const void *const *xs, const float *const *ts, int B, int H, int W,
                         float *grads, float *loss) {
    if (!net || !xs || !ts) return GABP_ERR_ARG;
    int rc = grad_impl(net, xs, ts, B, H, W, loss);
    if (rc) return rc;
    if (grads) WK(cudaMemcpy(grads, net->g, sizeof(float) * net->nparam, cudaMemcpyDefault), "copy grads");
    return GABP_OK;
}

int gabp_wsnet_train_step(gabp_wsnet *net, const void *const *xs, const float *const *ts, int B, int H, int W,
                          float lr, float *loss) {
    if (!net || !xs || !ts || !(lr > 0.f)) return GABP_ERR_ARG;
    int rc = grad_impl(net, xs, ts, B, H, W, loss);
    if (rc) return rc;
    net->step += 1;
    WK(gabp::nn::adam(net->w, net->m, net->v, net->g, net->nparam, lr, 0.9f, 0.999f, 1e-8f, net->step, net->w16,
                      net->stream),
       "adam");
    net->packed = false;
    WK(cudaStreamSynchronize(net->stream), "sync");
    return GABP_OK;
}

const char *gabp_wsnet_last_error(const gabp_wsnet *net) { return net ? net->err.c_str() : t_ws_err.c_str(); }

void gabp_wsnet_destroy(gabp_wsnet *net) {
    if (!net) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(net->dev);
    if (net->stream) cudaStreamSynchronize(net->stream);
    free_acts(net);
    cudaFree(net->w);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->g);
    cudaFree(net->w16);
    cudaFree(net->wt);
    cudaFree(net->wpk);
    cudaFree(net->wtpk);
    cudaFree(net->zbias);
    cudaFree(net->derr);
    if (net->stream) cudaStreamDestroy(net->stream);
    if (prev >= 0) cudaSetDevice(prev);
    delete net;
}

}  // extern "C"
