// Device-side arithmetic of one GaBP iteration, shared by the split and fused kernels.
//
// Message layout in HBM (both precisions, T = float or double):
//   prior messages: 5 planes of n (eta, Lambda) pairs, "outgoing" order: plane d at cell c
//     holds the message from the factor of cell c to node c + off_d, d = C, W, E, S, N
//     (off = 0, -1, +1, -nx, +nx).  Slots whose neighbour does not exist hold (0, 0).
//   observation messages: per observation (sorted by base cell), 8 values
//     eta_0..eta_3, Lambda_0..Lambda_3, one per bilinear corner.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gabp {

enum { DIR_C = 0, DIR_W = 1, DIR_E = 2, DIR_S = 3, DIR_N = 4 };

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using T2 = typename vec2<T>::type;

// Smallest normal number.
template <typename T> __device__ __forceinline__ T tiny_normal();
template <> __device__ __forceinline__ float tiny_normal<float>() { return 1.17549435e-38f; }
template <> __device__ __forceinline__ double tiny_normal<double>() { return 2.2250738585072014e-308; }

// Floor of a cavity precision relative to its slot's a^2 (see factor_messages).
template <typename T> __device__ __forceinline__ T lam_floor_rel();
template <> __device__ __forceinline__ float lam_floor_rel<float>() { return 1e-20f; }
template <> __device__ __forceinline__ double lam_floor_rel<double>() { return 1e-20; }

template <typename T> __device__ __forceinline__ T pos_inf();
template <> __device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double pos_inf<double>() {
    return __longlong_as_double(0x7ff0000000000000LL);
}

// Reciprocal.  FP32: the hardware approximation rcp.approx.ftz.f32, within 1 ulp over the
// range the callers use (they never pass 0, a denormal or an infinity: cavity precisions are
// floored at a normal number, and V is at least var > 0 and at most about 5e20).  FP64: IEEE
// division.
template <typename T> __device__ __forceinline__ T recip(T x);
template <> __device__ __forceinline__ float recip<float>(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }

// Explicitly rounded arithmetic for the message formulas: no multiply is contracted into a
// fused multiply-add unless written as one, so every kernel (scalar or packed two-lane FP32)
// evaluates them with the same roundings and produces the same bits.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Two-term compensated sum (TwoSum accumulation, Knuth TAOCP vol. 2 4.2.2): hi + lo carries
// the running sum to about twice the working precision.  Used for the belief sums so that
// the cavity (belief minus one message) keeps its relative accuracy even when that message
// dominates the belief.
template <typename T> struct CompSum {
    T hi, lo;
    __device__ __forceinline__ CompSum() : hi(T(0)), lo(T(0)) {}
    // start from a first term: identical to adding it to an empty sum (TwoSum(0, x) = (x, 0))
    __device__ __forceinline__ explicit CompSum(T first) : hi(first), lo(T(0)) {}
    __device__ __forceinline__ void add(T x) {
        T t = hi + x;
        T z = t - hi;
        T e = (hi - (t - z)) + (x - z);
        hi = t;
        lo += e;
    }
    // renormalise so that hi = fl(hi + lo)
    __device__ __forceinline__ void finish() {
        T t = hi + lo;
        lo = lo - (t - hi);
        hi = t;
    }
};

// A compensated belief: (eta_hi, eta_lo, lam_hi, lam_lo).
template <typename T> struct Belief {
    T ehi, elo, lhi, llo;
};

// Adds the observation messages into node (x, y) that come from the base cells of one row:
// base (x-1, row) with corner cl for indices [lo, mid) and base (x, row) with corner cr for
// [mid, hi).  The two ranges are adjacent in the base-sorted observation array, so the terms
// are added in increasing observation index; every iteration kernel uses this order (corners
// 1, 0 from the node's row, then 3, 2 from the row below).
template <typename T>
__device__ __forceinline__ void add_obs_pair(CompSum<T> &se, CompSum<T> &sl, const T *O, int lo, int mid,
                                             int hi, int cl, int cr) {
    for (int k = lo; k < hi; ++k) {
        const int c = k < mid ? cl : cr;
        se.add(O[8 * (int64_t)k + 2 * c]);
        sl.add(O[8 * (int64_t)k + 2 * c + 1]);
    }
}

// Cavity of one edge: the belief minus the edge's own incoming message, evaluated as
// (hi - own) + lo (App. A, variable-to-factor message).
template <typename T>
__device__ __forceinline__ void cavity(const Belief<T> &b, T own_eta, T own_lam, T &eta_c, T &lam_c) {
    lam_c = (b.lhi - own_lam) + b.llo;
    eta_c = (b.ehi - own_eta) + b.elo;
}

// Factor-to-variable messages of a rank-1 factor exp(-(1/(2 var)) (a . x - r)^2) with K slots
// (App. A factor-to-variable message generalised to K variables): for every slot v
//   V_v = var + sum_{u != v} a_u^2 / lam_u,   m_v = r - sum_{u != v} a_u eta_u / lam_u,
//   Lambda_v = a_v^2 / V_v,                   eta_v = a_v m_v / V_v.
// Leave-one-out sums come from prefix and suffix sums (no "total minus own" cancellation).
// Slots with a_u = 0 are skipped.  A cavity precision below 1e-20 a_u^2 (zero and negative
// included; in FP32 also below the smallest normal number) is raised to that floor.  Such a
// cavity is in the limit lam -> 0 with finite information, the linear potential exp(eta x):
// the messages to the other slots then equal that limit, (-a_v eta_u / a_u, 0), to a relative
// 1e-20 V, and nothing overflows.  (Far from the observations the precision recursion drives
// some cavity precisions far below the FP32 range while their information stays finite;
// treating them as carrying no information would drop that information.)
template <typename T, int K>
__device__ __forceinline__ void factor_messages(const T (&a)[K], T var, T r, const T (&lam)[K],
                                                const T (&eta)[K], T (&L)[K], T (&E)[K]) {
    T t[K], p[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        if (a[u] == T(0)) {
            t[u] = T(0);
            p[u] = T(0);
        } else {
            const T a2 = mul_rn(a[u], a[u]);
            // fmax returns the other operand for a NaN one: a NaN cavity precision is floored
            const T fl = fmax(mul_rn(lam_floor_rel<T>(), a2), tiny_normal<T>());
            const T rl = recip(fmax(lam[u], fl));
            t[u] = mul_rn(a2, rl);
            p[u] = mul_rn(a[u], mul_rn(eta[u], rl));
        }
    }
    T preV[K], preM[K];
    preV[0] = var;
    preM[0] = T(0);
#pragma unroll
    for (int v = 1; v < K; ++v) {
        preV[v] = add_rn(preV[v - 1], t[v - 1]);
        preM[v] = add_rn(preM[v - 1], p[v - 1]);
    }
    T sufV = T(0), sufM = T(0);
#pragma unroll
    for (int v = K - 1; v >= 0; --v) {
        const T V = add_rn(preV[v], sufV);
        const T M = add_rn(preM[v], sufM);
        const T rV = recip(V);
        L[v] = mul_rn(mul_rn(a[v], a[v]), rV);
        E[v] = mul_rn(mul_rn(a[v], add_rn(r, -M)), rV);
        sufV = add_rn(sufV, t[v]);
        sufM = add_rn(sufM, p[v]);
    }
}

// Damped update m_t = beta m_{t-1} + (1 - beta) m_new, evaluated as the fused multiply-add
// m_new + beta (m_{t-1} - m_new).
template <typename T> __device__ __forceinline__ T damp(T old, T fresh, T beta) {
    return fma_rn(beta, add_rn(old, -fresh), fresh);
}

// Number of existing 4-neighbours of node (i, j).
__device__ __forceinline__ int grid_degree(int i, int j, int nx, int ny) {
    return (j > 0) + (j < nx - 1) + (i > 0) + (i < ny - 1);
}

}  // namespace gabp
