// Packed two-lane FP32 arithmetic on (eta, Lambda) pairs and the persistent tile schedule,
// shared by the FP32 tile kernels (gabp_fused_tma.cu: alpha = 2 prior; gabp_fused_l2.cu:
// alpha = 4 prior).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "gabp_device.cuh"

namespace gabp {
namespace tiles {

// Schedule of a single-problem launch: runs of `run` tiles (one tile column of a band of `run`
// tile rows; the last band may be shorter), run u = band * ntx + column, dealt round-robin over
// the G blocks; step_x = G % ntx and step_b = G / ntx advance a block to its next run.
struct TileRuns {
    int run, ntx, nty, step_x, step_b;
};

// A block's position on its schedule: run (cx, band), tile r of len in that run; len = 0 once
// the block has no run left.
struct TileWalk {
    int cx, band, r, len;
    __device__ __forceinline__ void start(int u, const TileRuns &tr) {
        cx = u % tr.ntx;
        band = u / tr.ntx;
        r = 0;
        len = max(0, min(tr.run, tr.nty - band * tr.run));
    }
    __device__ __forceinline__ void next(const TileRuns &tr) {
        if (++r < len) return;
        r = 0;
        cx += tr.step_x;
        band += tr.step_b;
        if (cx >= tr.ntx) {
            cx -= tr.ntx;
            ++band;
        }
        len = max(0, min(tr.run, tr.nty - band * tr.run));
    }
    __device__ __forceinline__ int ty(const TileRuns &tr) const { return band * tr.run + r; }
};

// ---- packed two-lane FP32 arithmetic on (eta, Lambda) pairs ----
// Every (eta, Lambda) pair goes through the same sequence of roundings as the scalar formulas
// in gabp_device.cuh (add_rn, mul_rn, fma_rn per component), so the results are bit-identical
// to the other kernels; one packed instruction issues both components.
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // packed a - b, one instruction
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Compensated (eta, Lambda) belief sums: TwoSum accumulation of both components at once.
struct CompSum2 {
    float2 hi, lo;
    __device__ __forceinline__ explicit CompSum2(float2 first) : hi(first), lo(f2(0.f, 0.f)) {}
    __device__ __forceinline__ void add(float2 x) {
        const float2 t = add2(hi, x);
        const float2 z = sub2(t, hi);
        const float2 e = add2(sub2(hi, sub2(t, z)), sub2(x, z));
        hi = t;
        lo = add2(lo, e);
    }
    __device__ __forceinline__ void finish() {
        const float2 t = add2(hi, lo);
        lo = sub2(lo, sub2(t, hi));
        hi = t;
    }
};

// A compensated belief: hi = (eta_hi, Lambda_hi), lo = (eta_lo, Lambda_lo).
struct Belief2 {
    float2 hi, lo;
};

// Cavity (belief minus the edge's own message), (hi - own) + lo per component.
__device__ __forceinline__ float2 cavity2(const Belief2 &b, float2 own) { return add2(sub2(b.hi, own), b.lo); }

// Observation messages into one node from the base cells of one row, in increasing
// observation index (the order every kernel uses): corner cl for [lo, mid), cr for [mid, hi).
__device__ __forceinline__ void add_obs_pair2(CompSum2 &s, const float *O, int lo, int mid, int hi, int cl, int cr) {
    for (int k = lo; k < hi; ++k) {
        const int c = k < mid ? cl : cr;
        s.add(*reinterpret_cast<const float2 *>(O + 8 * (int64_t)k + 2 * c));
    }
}

// Factor-to-variable messages of a rank-1 factor with K slots on (eta, Lambda) pairs: the
// arithmetic of factor_messages (App. A) with the (M, V) sums and the (eta, Lambda) outputs
// carried as pairs.  cav[u] = cavity (eta, Lambda) of slot u; out[u] = message (eta, Lambda).
// UNIT_A: every nonzero a_u^2 is at least 1.2e-18 (cell factors: -1 and kappa^2 + deg with
// deg >= 1, as on every grid of four or more columns), so 1e-20 a_u^2 is a normal number and the
// second floor of factor_messages is a no-op that can be left out.
template <int K, bool UNIT_A>
__device__ __forceinline__ void factor_messages2(const float (&a)[K], float var, float r, const float2 (&cav)[K],
                                                 float2 (&out)[K]) {
    float2 tp[K];   // (a eta / lam, a^2 / lam), lam floored as in factor_messages
#pragma unroll
    for (int u = 0; u < K; ++u) {
        if (a[u] == 0.f) {
            tp[u] = f2(0.f, 0.f);
        } else {
            const float a2 = mul_rn(a[u], a[u]);
            float fl = mul_rn(lam_floor_rel<float>(), a2);
            if (!UNIT_A) fl = fmaxf(fl, tiny_normal<float>());
            const float rl = recip(fmaxf(cav[u].y, fl));
            tp[u] = mul2(f2(a[u], a2), f2(mul_rn(cav[u].x, rl), rl));
        }
    }
    float2 pre[K];   // prefix sums (M, V), V starting from var
    pre[0] = f2(0.f, var);
#pragma unroll
    for (int v = 1; v < K; ++v) pre[v] = add2(pre[v - 1], tp[v - 1]);
    float2 suf = f2(0.f, 0.f);
#pragma unroll
    for (int v = K - 1; v >= 0; --v) {
        const float2 MV = add2(pre[v], suf);
        const float rV = recip(MV.y);
        out[v] = mul2(f2(mul_rn(a[v], add_rn(r, -MV.x)), mul_rn(a[v], a[v])), f2(rV, rV));
        suf = add2(suf, tp[v]);
    }
}

// Damped update of an (eta, Lambda) pair: fresh + beta (old - fresh) as one fused multiply-add.
__device__ __forceinline__ float2 damp2(float2 old, float2 fresh, float2 beta2) {
    return fma2(beta2, sub2(old, fresh), fresh);
}

// Update of observation factor k (bilinear interpolation weights, var = sigma^2, r = y; App. A):
// cavities of its four corner nodes from their compensated beliefs bn[u], the factor-to-variable
// messages, damping, and the store of the four new messages.  Wt: 4 weights per observation; YV:
// (y, sigma^2) per observation; O / OQ: the observation messages of the current / next buffer,
// (eta, Lambda) of corners 0..3 interleaved.
__device__ __forceinline__ void obs_factor2(const Belief2 *const (&bn)[4], const float *Wt, const float *YV,
                                            const float *O, float *OQ, int64_t k, float2 beta2) {
    const float4 w4 = *reinterpret_cast<const float4 *>(Wt + 4 * k);
    const float aw[4] = {w4.x, w4.y, w4.z, w4.w};
    const float4 o01 = *reinterpret_cast<const float4 *>(O + 8 * k);   // (eta, Lambda) x 2
    const float4 o23 = *reinterpret_cast<const float4 *>(O + 8 * k + 4);
    float2 own4[4] = {f2(o01.x, o01.y), f2(o01.z, o01.w), f2(o23.x, o23.y), f2(o23.z, o23.w)}, cav[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) cav[u] = cavity2(*bn[u], own4[u]);
    const float2 yv = *reinterpret_cast<const float2 *>(YV + 2 * k);
    float2 msg[4];
    factor_messages2<4, false>(aw, yv.y, yv.x, cav, msg);
#pragma unroll
    for (int u = 0; u < 4; ++u) msg[u] = damp2(own4[u], msg[u], beta2);
    *reinterpret_cast<float4 *>(OQ + 8 * k) = make_float4(msg[0].x, msg[0].y, msg[1].x, msg[1].y);
    *reinterpret_cast<float4 *>(OQ + 8 * k + 4) = make_float4(msg[2].x, msg[2].y, msg[3].x, msg[3].y);
}

}  // namespace tiles
}  // namespace gabp
