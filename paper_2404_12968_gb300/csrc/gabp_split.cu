// Split GaBP iteration (three kernels: beliefs, prior factors, observation factors) and the
// auxiliary kernels: message initialisation, FP64 observation precompute, FP64 residual and
// marginals.  The split iteration is the plain form of one synchronous iteration; the fused
// kernel (gabp_fused.cu) computes the same messages in one pass.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "gabp_device.cuh"
#include "gabp_internal.h"
#include "gabp_l2.cuh"

namespace gabp {

namespace {

constexpr int TPB = 256;

template <typename T> struct __align__(4 * sizeof(T)) BeliefStore {
    T ehi, elo, lhi, llo;
};

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }

inline unsigned nblocks(int64_t count) { return (unsigned)((count + TPB - 1) / TPB); }

// Grid coordinates (row i, column j) of node v: a 32-bit division while the index fits (a 64-bit
// division is a long instruction sequence)
__device__ __forceinline__ void node_rc(int64_t v, int nx, int &i, int &j) {
    if (v <= 0x7fffffff) {
        const unsigned q = (unsigned)v / (unsigned)nx;
        i = (int)q;
        j = (int)((unsigned)v - q * (unsigned)nx);
    } else {
        i = (int)(v / nx);
        j = (int)(v - (int64_t)i * nx);
    }
}
// Row-wise launch over an nx x ny grid: blocks of TPB columns of one row (no division on the
// device), rows strided by gridDim.y (at most 65535)
inline dim3 row_grid(int nx, int ny) { return dim3((unsigned)((nx + TPB - 1) / TPB), (unsigned)std::min(ny, 65535)); }

// ---- beliefs (App. A, state update): sum of every incoming message, compensated ----
// compensated belief of node v = (i, j) from the messages of buffer src
template <typename T> __device__ __forceinline__ BeliefStore<T> node_belief(const DevProblem &p, int64_t v, int i, int j, int src) {
    const int nx = p.nx, ny = p.ny;
    const T2<T> *P = (const T2<T> *)p.P[src];
    const T *O = (const T *)p.O[src];
    const int64_t pn = p.pn, pv = plane_at(p, i, j);
    T2<T> q = P[DIR_C * pn + pv];
    CompSum<T> se(q.x), sl(q.y);
    if (j > 0) { q = P[DIR_E * pn + pv - 1]; se.add(q.x); sl.add(q.y); }
    if (j < nx - 1) { q = P[DIR_W * pn + pv + 1]; se.add(q.x); sl.add(q.y); }
    if (i > 0) { q = P[DIR_N * pn + pv - p.px]; se.add(q.x); sl.add(q.y); }
    if (i < ny - 1) { q = P[DIR_S * pn + pv + p.px]; se.add(q.x); sl.add(q.y); }
    if (p.m > 0) {
        const int *optr = p.optr;
        // bases (j-1, i), (j, i) then (j-1, i-1), (j, i-1): corners 1, 0, 3, 2
        add_obs_pair(se, sl, O, j > 0 ? optr[v - 1] : optr[v], optr[v], optr[v + 1], 1, 0);
        if (i > 0) add_obs_pair(se, sl, O, j > 0 ? optr[v - nx - 1] : optr[v - nx], optr[v - nx], optr[v - nx + 1], 3, 2);
    }
    se.finish();
    sl.finish();
    BeliefStore<T> b;
    b.ehi = se.hi; b.elo = se.lo; b.lhi = sl.hi; b.llo = sl.lo;
    return b;
}

template <typename T> __global__ void k_beliefs(DevProblem p, int src) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    ((BeliefStore<T> *)p.belief)[v] = node_belief<T>(p, v, i, j, src);
}

template <typename T> __device__ __forceinline__ Belief<T> load_belief(const DevProblem &p, int64_t v) {
    BeliefStore<T> s = ((const BeliefStore<T> *)p.belief)[v];
    Belief<T> b;
    b.ehi = s.ehi; b.elo = s.elo; b.lhi = s.lhi; b.llo = s.llo;
    return b;
}

// ---- prior cell factors: a = row c of L over (C, W, E, S, N), var = 1/gamma, r = 0 ----
template <typename T> __global__ void k_prior(DevProblem p, int src, T beta) {
    const int64_t c = gtid();
    if (c >= p.n) return;
    const int nx = p.nx, ny = p.ny;
    int i, j;
    node_rc(c, nx, i, j);
    const int64_t pn = p.pn, pc = plane_at(p, i, j);
    const T2<T> *P = (const T2<T> *)p.P[src];
    T2<T> *Q = (T2<T> *)p.P[src ^ 1];
    const int deg = grid_degree(i, j, nx, ny);
    const T a[5] = {cell_coef<T>(p, deg), j > 0 ? T(-1) : T(0), j < nx - 1 ? T(-1) : T(0),
                    i > 0 ? T(-1) : T(0), i < ny - 1 ? T(-1) : T(0)};
    const int64_t node[5] = {c, c - 1, c + 1, c - nx, c + nx};
    T2<T> own[5];
    T lam[5], eta[5];
#pragma unroll
    for (int u = 0; u < 5; ++u) {
        own[u] = P[u * pn + pc];
        if (a[u] != T(0)) {
            cavity(load_belief<T>(p, node[u]), own[u].x, own[u].y, eta[u], lam[u]);
        } else {
            lam[u] = T(1);
            eta[u] = T(0);
        }
    }
    T L[5], E[5];
    const T r = p.ptgt ? ((const T *)p.ptgt)[c] : T(0);
    factor_messages<T, 5>(a, prior_var<T>(p), r, lam, eta, L, E);
#pragma unroll
    for (int u = 0; u < 5; ++u) {
        T2<T> out;
        if (a[u] != T(0)) {
            out.x = damp(own[u].x, E[u], beta);
            out.y = damp(own[u].y, L[u], beta);
        } else {
            out.x = T(0);
            out.y = T(0);
        }
        Q[u * pn + pc] = out;
    }
}

// ---- the alpha = 4 prior (coefficients and slot offsets in gabp_l2.cuh) ----
// beliefs of order-2 contexts: node v receives slot d of the factor of cell v - offset(d),
// summed in slot order, then the observation messages as for order 1
template <typename T, bool INTERIOR> __device__ __forceinline__ void beliefs_l2(const DevProblem &p, int64_t v, int i, int j, int src) {
    const int nx = p.nx, ny = p.ny;
    const T2<T> *P = (const T2<T> *)p.P[src];
    const T *O = (const T *)p.O[src];
    const int64_t n = p.n;
    T2<T> q = P[v];
    CompSum<T> se(q.x), sl(q.y);
#pragma unroll
    for (int d = 1; d < L2_SLOTS; ++d) {
        const int ci = i - l2_dy(d), cj = j - l2_dx(d);
        if (INTERIOR || (ci >= 0 && ci < ny && cj >= 0 && cj < nx)) {
            q = P[d * n + v - ((int64_t)l2_dy(d) * nx + l2_dx(d))];
            se.add(q.x);
            sl.add(q.y);
        }
    }
    if (p.m > 0) {
        const int *optr = p.optr;
        add_obs_pair(se, sl, O, j > 0 ? optr[v - 1] : optr[v], optr[v], optr[v + 1], 1, 0);
        if (i > 0) add_obs_pair(se, sl, O, j > 0 ? optr[v - nx - 1] : optr[v - nx], optr[v - nx], optr[v - nx + 1], 3, 2);
    }
    se.finish();
    sl.finish();
    BeliefStore<T> b;
    b.ehi = se.hi; b.elo = se.lo; b.lhi = sl.hi; b.llo = sl.lo;
    ((BeliefStore<T> *)p.belief)[v] = b;
}

template <typename T> __global__ void k_beliefs_l2(DevProblem p, int src) {
    const int nx = p.nx, ny = p.ny;
    const int j = blockIdx.x * TPB + threadIdx.x;
    if (j >= nx) return;
    for (int i = blockIdx.y; i < ny; i += gridDim.y) {
        const int64_t v = (int64_t)i * nx + j;
        if (i >= 2 && i < ny - 2 && j >= 2 && j < nx - 2) beliefs_l2<T, true>(p, v, i, j, src);
        else beliefs_l2<T, false>(p, v, i, j, src);
    }
}

// order-2 cell factors: a = row c of L^2, var = 1/gamma, r = 0
template <typename T, bool INTERIOR>
__device__ __forceinline__ void prior_l2(const DevProblem &p, int64_t c, int i, int j, int src, T beta) {
    const int nx = p.nx;
    const int64_t n = p.n;
    const T2<T> *P = (const T2<T> *)p.P[src];
    T2<T> *Q = (T2<T> *)p.P[src ^ 1];
    T a[L2_SLOTS], lam[L2_SLOTS], eta[L2_SLOTS];
    T2<T> own[L2_SLOTS];
#pragma unroll
    for (int d = 0; d < L2_SLOTS; ++d) {
        a[d] = l2_coef_t<T, INTERIOR>(p, i, j, d);
        own[d] = P[d * n + c];
        if (INTERIOR || a[d] != T(0)) {
            cavity(load_belief<T>(p, c + (int64_t)l2_dy(d) * nx + l2_dx(d)), own[d].x, own[d].y, eta[d], lam[d]);
        } else {
            lam[d] = T(1);
            eta[d] = T(0);
        }
    }
    T L[L2_SLOTS], E[L2_SLOTS];
    factor_messages<T, L2_SLOTS>(a, prior_var<T>(p), T(0), lam, eta, L, E);
#pragma unroll
    for (int d = 0; d < L2_SLOTS; ++d) {
        T2<T> out;
        if (INTERIOR || a[d] != T(0)) {
            out.x = damp(own[d].x, E[d], beta);
            out.y = damp(own[d].y, L[d], beta);
        } else {
            out.x = T(0);
            out.y = T(0);
        }
        Q[d * n + c] = out;
    }
}

// (FP32: registers bounded for 3 resident blocks of 256 threads per SM, measured 3.5 % faster
// than the unbounded 103)
template <typename T> __global__ void __launch_bounds__(TPB, sizeof(T) == 4 ? 3 : 1)
    k_prior_l2(DevProblem p, int src, T beta) {
    const int nx = p.nx, ny = p.ny;
    const int j = blockIdx.x * TPB + threadIdx.x;
    if (j >= nx) return;
    for (int i = blockIdx.y; i < ny; i += gridDim.y) {
        const int64_t c = (int64_t)i * nx + j;
        if (i >= 2 && i < ny - 2 && j >= 2 && j < nx - 2) prior_l2<T, true>(p, c, i, j, src, beta);
        else prior_l2<T, false>(p, c, i, j, src, beta);
    }
}

// cold / paper initialisation of the 13 planes (as k_init_prior)
template <typename T> __global__ void k_init_prior_l2(DevProblem p, int dst, int paper) {
    const int64_t c = gtid();
    if (c >= p.n) return;
    const int nx = p.nx;
    int i, j;
    node_rc(c, nx, i, j);
    T2<T> *Q = (T2<T> *)p.P[dst];
#pragma unroll
    for (int d = 0; d < L2_SLOTS; ++d) {
        const double a = l2_coef(p, i, j, d);
        T2<T> o;
        o.x = T(0);
        o.y = a == 0.0 ? T(0) : (paper ? T(1e-8) : T(p.gamma * a * a));
        Q[d * p.n + c] = o;
    }
}

// ---- observation factors: a = bilinear weights, var = sigma^2, r = y ----
template <typename T> __global__ void k_obs(DevProblem p, int src, T beta) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    const int nx = p.nx;
    const int64_t b = p.obase[k];
    const T *W = (const T *)p.ow;
    const T *YV = (const T *)p.ovar;
    const T *O = (const T *)p.O[src];
    T *Q = (T *)p.O[src ^ 1];
    const T a[4] = {W[4 * k], W[4 * k + 1], W[4 * k + 2], W[4 * k + 3]};
    const int64_t node[4] = {b, b + 1, b + nx, b + nx + 1};
    T oe[4], ol[4], lam[4], eta[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        oe[u] = O[8 * k + 2 * u];
        ol[u] = O[8 * k + 2 * u + 1];
        cavity(load_belief<T>(p, node[u]), oe[u], ol[u], eta[u], lam[u]);
    }
    T L[4], E[4];
    factor_messages<T, 4>(a, YV[2 * k + 1], YV[2 * k], lam, eta, L, E);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        Q[8 * k + 2 * u] = damp(oe[u], E[u], beta);
        Q[8 * k + 2 * u + 1] = damp(ol[u], L[u], beta);
    }
}

// ---- initialisation ----
template <typename T> __global__ void k_init_prior(DevProblem p, int dst, int paper) {
    const int64_t c = gtid();
    if (c >= p.n) return;
    const int nx = p.nx, ny = p.ny;
    int i, j;
    node_rc(c, nx, i, j);
    const int deg = grid_degree(i, j, nx, ny);
    const bool has[5] = {true, j > 0, j < nx - 1, i > 0, i < ny - 1};
    T2<T> *Q = (T2<T> *)p.P[dst];
#pragma unroll
    for (int u = 0; u < 5; ++u) {
        T2<T> o;
        o.x = T(0);
        T cold;   // gamma a_u^2: FP32 from the host-rounded table (no FP64 instruction)
        if constexpr (sizeof(T) == 4) cold = u == 0 ? p.init_c_f[deg] : p.init_n_f;
        else cold = u == 0 ? p.gamma * p.aC[deg] * p.aC[deg] : p.gamma * -1.0 * -1.0;
        o.y = !has[u] ? T(0) : (paper ? T(1e-8) : cold);
        Q[u * p.pn + plane_at(p, i, j)] = o;
    }
}

template <typename T> __global__ void k_init_obs(DevProblem p, int dst, int paper) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    T *Q = (T *)p.O[dst];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const double w = p.ow64[4 * k + u];
        Q[8 * k + 2 * u] = T(0);
        Q[8 * k + 2 * u + 1] = paper ? T(1e-8) : T(p.oys64[2 * k + 1] * w * w);
    }
}

// number of factor slots touching node v (prior factors + observation corners)
__device__ __forceinline__ int node_slots(const DevProblem &p, int64_t v) {
    const int nx = p.nx, ny = p.ny;
    int i, j;
    node_rc(v, nx, i, j);
    int d = 1 + grid_degree(i, j, nx, ny);
    if (p.m > 0) {
        const int *o = p.optr;
        d += o[v + 1] - o[v];
        if (j > 0) d += o[v] - o[v - 1];
        if (i > 0) d += o[v - nx + 1] - o[v - nx];
        if (i > 0 && j > 0) d += o[v - nx] - o[v - nx - 1];
    }
    return d;
}

template <typename T>
__global__ void k_init_warm_prior(DevProblem p, int dst, const double *mu0, const double *lam0) {
    const int64_t c = gtid();
    if (c >= p.n) return;
    const int nx = p.nx, ny = p.ny;
    int i, j;
    node_rc(c, nx, i, j);
    const bool exists[5] = {true, j > 0, j < nx - 1, i > 0, i < ny - 1};
    const int64_t node[5] = {c, c - 1, c + 1, c - nx, c + nx};
    T2<T> *Q = (T2<T> *)p.P[dst];
#pragma unroll
    for (int u = 0; u < 5; ++u) {
        T2<T> o;
        o.x = T(0);
        o.y = T(0);
        if (exists[u]) {
            const double L = lam0[node[u]] / (double)node_slots(p, node[u]);
            o.x = T(mu0[node[u]] * L);
            o.y = T(L);
        }
        Q[u * p.pn + plane_at(p, i, j)] = o;
    }
}

template <typename T>
__global__ void k_init_warm_obs(DevProblem p, int dst, const double *mu0, const double *lam0) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    const int64_t b = p.obase[k];
    const int64_t node[4] = {b, b + 1, b + p.nx, b + p.nx + 1};
    T *Q = (T *)p.O[dst];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const double L = lam0[node[u]] / (double)node_slots(p, node[u]);
        Q[8 * k + 2 * u] = T(mu0[node[u]] * L);
        Q[8 * k + 2 * u + 1] = T(L);
    }
}

// ---- FP64 observation precompute (the factor precompute of the observation factors) ----
template <typename T>
__global__ void k_obs_precompute(DevProblem p, const double *xy, const double *yv, const double *var) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    const int nx = p.nx;
    const int b = p.obase[k];
    const int i0 = b / nx, j0 = b - i0 * nx;
    const double fu = xy[2 * k] - (double)j0;
    const double fv = xy[2 * k + 1] - (double)i0;
    const double w[4] = {(1.0 - fu) * (1.0 - fv), fu * (1.0 - fv), (1.0 - fu) * fv, fu * fv};
    T *W = (T *)p.ow;
    T *YV = (T *)p.ovar;
    double *W64 = (double *)p.ow64;
    double *YS64 = (double *)p.oys64;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        W[4 * k + u] = T(w[u]);
        W64[4 * k + u] = w[u];
    }
    YV[2 * k] = T(yv[k]);
    YV[2 * k + 1] = T(var[k]);
    YS64[2 * k] = yv[k];
    YS64[2 * k + 1] = 1.0 / var[k];
}

// ---- per-cell observation index: optr[c] = lower bound of c in the sorted base cells ----
__global__ void k_obs_pointers(DevProblem p) {
    const int64_t c = gtid();
    if (c > p.n) return;
    int64_t lo = 0, hi = p.m;   // first k with obase[k] >= c
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (p.obase[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    ((int *)p.optr)[c] = (int)lo;
}

// ---- deterministic FP64 reductions: fixed grid, fixed per-thread order, smem tree ----
__device__ __forceinline__ double block_sum(double x) {
    __shared__ double sh[TPB];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    return sh[0];
}

__global__ void k_final_sum(const double *part, int count, double *out) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < count; q += TPB) acc += part[q];
    double s = block_sum(acc);
    if (threadIdx.x == 0) *out = s;
}

// sum over observation edges into node v of w_kc * val_k (FP64), corners in fixed order
__device__ __forceinline__ double obs_gather64(const DevProblem &p, int64_t v, int i, int j,
                                               const double *val, int stride, int off) {
    const int nx = p.nx;
    const int *o = p.optr;
    double acc = 0.0;
    for (int k = o[v]; k < o[v + 1]; ++k) acc += p.ow64[4 * (int64_t)k + 0] * val[stride * (int64_t)k + off];
    if (j > 0)
        for (int k = o[v - 1]; k < o[v]; ++k) acc += p.ow64[4 * (int64_t)k + 1] * val[stride * (int64_t)k + off];
    if (i > 0)
        for (int k = o[v - nx]; k < o[v - nx + 1]; ++k) acc += p.ow64[4 * (int64_t)k + 2] * val[stride * (int64_t)k + off];
    if (i > 0 && j > 0)
        for (int k = o[v - nx - 1]; k < o[v - nx]; ++k) acc += p.ow64[4 * (int64_t)k + 3] * val[stride * (int64_t)k + off];
    return acc;
}

// (L x)_v = (kappa^2 + deg) x_v - sum of existing neighbours
__device__ __forceinline__ double apply_L(const DevProblem &p, const double *x, int64_t v, int i, int j) {
    const int nx = p.nx, ny = p.ny;
    double s = p.aC[grid_degree(i, j, nx, ny)] * x[v];
    if (j > 0) s -= x[v - 1];
    if (j < nx - 1) s -= x[v + 1];
    if (i > 0) s -= x[v - nx];
    if (i < ny - 1) s -= x[v + nx];
    return s;
}

// ||b||^2 with b_v = sum over incoming observation edges of w * s * y, plus gamma (L r)_v for
// cell-factor targets r
__global__ void k_rhs_norm(DevProblem p) {
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t v = gtid(); v < p.n; v += stride) {
        int i, j;
        node_rc(v, p.nx, i, j);
        double bv = 0.0;
        if (p.m > 0) {
            // w * (s * y): gather w_kc * y_k * s_k
            const int *o = p.optr;
            const int nx = p.nx;
            for (int k = o[v]; k < o[v + 1]; ++k) bv += p.ow64[4 * (int64_t)k] * p.oys64[2 * (int64_t)k] * p.oys64[2 * (int64_t)k + 1];
            if (j > 0)
                for (int k = o[v - 1]; k < o[v]; ++k) bv += p.ow64[4 * (int64_t)k + 1] * p.oys64[2 * (int64_t)k] * p.oys64[2 * (int64_t)k + 1];
            if (i > 0)
                for (int k = o[v - nx]; k < o[v - nx + 1]; ++k) bv += p.ow64[4 * (int64_t)k + 2] * p.oys64[2 * (int64_t)k] * p.oys64[2 * (int64_t)k + 1];
            if (i > 0 && j > 0)
                for (int k = o[v - nx - 1]; k < o[v - nx]; ++k) bv += p.ow64[4 * (int64_t)k + 3] * p.oys64[2 * (int64_t)k] * p.oys64[2 * (int64_t)k + 1];
        }
        if (p.ptgt64) bv += p.gamma * apply_L(p, p.ptgt64, v, i, j);   // gamma L^T r (L symmetric)
        acc += bv * bv;
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0) p.part[blockIdx.x] = s;
}

// ---- the residual of FP32 contexts in double-float arithmetic ----
// A value is an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2), about 48 significant
// bits.  Error-free transformations: TwoSum (Knuth), Fast2Sum (Dekker, |a| >= |b|) and the
// product error by fused multiply-add; every operation is explicitly rounded.  It replaces FP64
// arithmetic, whose throughput on this GPU is a small fraction of FP32's.
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl df_fast2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    const float s = __fadd_rn(x.hi, y.hi);
    const float bb = __fsub_rn(s, x.hi);
    const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    return df_fast2sum(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast2sum(p, e);
}
__device__ __forceinline__ dfl df_ld(const float2 *a, int64_t i) {
    const float2 v = a[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void df_st(float2 *a, int64_t i, dfl x) { a[i] = make_float2(x.hi, x.lo); }
__device__ __forceinline__ dfl df_split(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}

__global__ void k_df_precompute(DevProblem p) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    float2 *w = (float2 *)p.owdf;
    float2 *ys = (float2 *)p.oysdf;
#pragma unroll
    for (int c = 0; c < 4; ++c) df_st(w, 4 * k + c, df_split(p.ow64[4 * k + c]));
    df_st(ys, 2 * k, df_split(p.oys64[2 * k]));
    df_st(ys, 2 * k + 1, df_split(p.oys64[2 * k + 1]));
}

// mu = eta / Lambda from the compensated FP32 belief (hi + lo pairs): quotient of the leading
// parts, one correction with the exact remainder eta - Lambda q1
// mu = eta / Lambda of a compensated FP32 belief as a double-float pair: the quotient of the
// leading parts plus one correction from the exact remainder eta - Lambda q1
__device__ __forceinline__ dfl df_belief_mean(const BeliefStore<float> &b) {
    const dfl eta = {b.ehi, b.elo}, lam = {b.lhi, b.llo};
    const float q1 = __fdiv_rn(eta.hi, lam.hi);
    const dfl r = df_add(eta, df_neg(df_mul(lam, {q1, 0.f})));
    const float q2 = __fdiv_rn(r.hi, lam.hi);
    return df_fast2sum(q1, q2);
}

// the same mean straight from the messages of buffer src (the belief kept in registers, not
// stored): the FP32 residual's first pass
__global__ void k_mu_direct_df(DevProblem p, int src) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    df_st((float2 *)p.mu64, v, df_belief_mean(node_belief<float>(p, v, i, j, src)));
}

// e_k = s_k (h_k . mu - y_k)
__global__ void k_obs_err_df(DevProblem p) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    const int64_t b = p.obase[k];
    const float2 *mu = (const float2 *)p.mu64;
    const int64_t nodes[4] = {b, b + 1, b + p.nx, b + p.nx + 1};
    dfl hm = df_mul(df_ld(p.owdf, 4 * k), df_ld(mu, nodes[0]));
#pragma unroll
    for (int c = 1; c < 4; ++c) hm = df_add(hm, df_mul(df_ld(p.owdf, 4 * k + c), df_ld(mu, nodes[c])));
    const dfl e = df_mul(df_ld(p.oysdf, 2 * k + 1), df_add(hm, df_neg(df_ld(p.oysdf, 2 * k))));
    df_st((float2 *)p.e64, k, e);
}

// (L x)_v with the zero-Neumann stencil: (kappa^2 + deg) x_v - sum of the existing neighbours
__device__ __forceinline__ dfl apply_L_df(const DevProblem &p, const float2 *x, int64_t v, int i, int j) {
    const int nx = p.nx, ny = p.ny;
    const int d = grid_degree(i, j, nx, ny);
    dfl s = df_mul({p.aC_f[d], p.aC_lo[d]}, df_ld(x, v));
    if (j > 0) s = df_add(s, df_neg(df_ld(x, v - 1)));
    if (j < nx - 1) s = df_add(s, df_neg(df_ld(x, v + 1)));
    if (i > 0) s = df_add(s, df_neg(df_ld(x, v - nx)));
    if (i < ny - 1) s = df_add(s, df_neg(df_ld(x, v + nx)));
    return s;
}

__global__ void k_Lmu_df(DevProblem p) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    dfl z = apply_L_df(p, (const float2 *)p.mu64, v, i, j);
    if (p.ptgtdf) z = df_add(z, df_neg(df_ld(p.ptgtdf, v)));   // l_v . mu - r_v
    df_st((float2 *)p.z64, v, z);
}

// partial sums of r_v^2, r = b - A mu = -gamma L (L mu) - H^T (s (H mu - y)); per-thread sums in
// double-float, then the same fixed-order FP64 block reduction as the FP64 path
__global__ void k_res_df(DevProblem p) {
    dfl acc = {0.f, 0.f};
    const int64_t stride = (int64_t)gridDim.x * TPB;
    const float2 *e = (const float2 *)p.e64;
    const int *o = p.optr;
    const int nx = p.nx;
    for (int64_t v = gtid(); v < p.n; v += stride) {
        int i, j;
        node_rc(v, nx, i, j);
        dfl r = df_neg(df_mul({p.gam_hi, p.gam_lo}, apply_L_df(p, (const float2 *)p.z64, v, i, j)));
        if (p.m > 0) {
            for (int k = o[v]; k < o[v + 1]; ++k) r = df_add(r, df_neg(df_mul(df_ld(p.owdf, 4 * (int64_t)k), df_ld(e, k))));
            if (j > 0)
                for (int k = o[v - 1]; k < o[v]; ++k)
                    r = df_add(r, df_neg(df_mul(df_ld(p.owdf, 4 * (int64_t)k + 1), df_ld(e, k))));
            if (i > 0)
                for (int k = o[v - nx]; k < o[v - nx + 1]; ++k)
                    r = df_add(r, df_neg(df_mul(df_ld(p.owdf, 4 * (int64_t)k + 2), df_ld(e, k))));
            if (i > 0 && j > 0)
                for (int k = o[v - nx - 1]; k < o[v - nx]; ++k)
                    r = df_add(r, df_neg(df_mul(df_ld(p.owdf, 4 * (int64_t)k + 3), df_ld(e, k))));
        }
        acc = df_add(acc, df_mul(r, r));
    }
    double s = block_sum((double)acc.hi + (double)acc.lo);
    if (threadIdx.x == 0) p.part[blockIdx.x] = s;
}

template <typename T> __global__ void k_mu(DevProblem p) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    const BeliefStore<T> b = ((const BeliefStore<T> *)p.belief)[v];
    p.mu64[v] = ((double)b.ehi + (double)b.elo) / ((double)b.lhi + (double)b.llo);
}

__global__ void k_obs_err(DevProblem p) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    const int64_t b = p.obase[k];
    const double *w = p.ow64 + 4 * k;
    const double hm = w[0] * p.mu64[b] + w[1] * p.mu64[b + 1] + w[2] * p.mu64[b + p.nx] +
                      w[3] * p.mu64[b + p.nx + 1];
    p.e64[k] = p.oys64[2 * k + 1] * (hm - p.oys64[2 * k]);
}

// y = L x (FP64); the alpha = 4 residual applies L four times
__global__ void k_Lx(DevProblem p, const double *x, double *y) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    y[v] = apply_L(p, x, v, i, j);
}

__global__ void k_Lmu(DevProblem p) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    double z = apply_L(p, p.mu64, v, i, j);
    if (p.ptgt64) z -= p.ptgt64[v];   // l_v . mu - r_v
    p.z64[v] = z;
}

// r = b - A mu = -gamma L (L mu) - H^T S (H mu - y); accumulate ||r||^2
__global__ void k_res(DevProblem p) {
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t v = gtid(); v < p.n; v += stride) {
        int i, j;
        node_rc(v, p.nx, i, j);
        double r = -p.gamma * apply_L(p, p.z64, v, i, j);
        if (p.m > 0) r -= obs_gather64(p, v, i, j, p.e64, 1, 0);
        acc += r * r;
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0) p.part[blockIdx.x] = s;
}

// marginal mean (and variance) of node v from its compensated belief
template <typename T>
__device__ __forceinline__ void marg_from_belief(const BeliefStore<T> &b, int64_t v, double *mean, double *var) {
    if constexpr (sizeof(T) == 4) {
        // FP32 beliefs (hi + lo pairs): the mean as the residual forms it, a double-float
        // quotient with one correction from the exact remainder, widened to FP64 once (no FP64
        // division: FP64 throughput is a small fraction of FP32 here)
        const dfl q = df_belief_mean(b);
        mean[v] = (double)q.hi + (double)q.lo;
        if (var) var[v] = 1.0 / ((double)b.lhi + (double)b.llo);
    } else {
        const double L = (double)b.lhi + (double)b.llo;
        mean[v] = ((double)b.ehi + (double)b.elo) / L;
        if (var) var[v] = 1.0 / L;
    }
}

// the marginals straight from the messages of buffer src (the belief formed in registers)
template <typename T> __global__ void k_marg(DevProblem p, int src, double *mean, double *var) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    marg_from_belief<T>(node_belief<T>(p, v, i, j, src), v, mean, var);
}

// the marginals from the stored beliefs (the alpha = 4 prior's beliefs come from k_beliefs_l2)
template <typename T> __global__ void k_marg_stored(DevProblem p, double *mean, double *var) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    marg_from_belief<T>(((const BeliefStore<T> *)p.belief)[v], v, mean, var);
}

// ---- learned warm start: network inputs, training targets, decoded initial beliefs ----
// Grid padded to Hp x Wp (multiples of 8); node (i, j) -> pixel (i, j).

// x[i][j][0..15]: mean of y / scale over the observations whose nearest node is (i, j), the
// mask of such nodes, log(kappa) + 3, zeros.  The nearest node of an observation is the corner
// of its base cell nearest to it along each axis, found from the fractions fu = w1 + w3 and
// fv = w2 + w3 (a fraction of exactly 0.5 goes to the higher index).
template <typename T>
__global__ void k_ws_input(DevProblem p, T inv_scale, float kfeat, int Hp, int Wp, __nv_bfloat16 *x) {
    const int64_t q = gtid();
    if (q >= (int64_t)Hp * Wp) return;
    int i, j;
    node_rc(q, Wp, i, j);
    const T *ow = (const T *)p.ow;    // 4 weights per observation
    const T *oyv = (const T *)p.ovar; // (y, variance) per observation
    T sum = T(0);
    int cnt = 0;
    if (i < p.ny && j < p.nx && p.m > 0) {
        const int nx = p.nx;
        const int64_t v = (int64_t)i * nx + j;
        const int64_t bases[4] = {v, v - 1, v - nx, v - nx - 1};
        const bool ok[4] = {true, j > 0, i > 0, i > 0 && j > 0};
        for (int c = 0; c < 4; ++c) {
            if (!ok[c]) continue;
            for (int k = p.optr[bases[c]]; k < p.optr[bases[c] + 1]; ++k) {
                const T *w = ow + 4 * (int64_t)k;
                const int near = (w[1] + w[3] >= T(0.5) ? 1 : 0) + (w[2] + w[3] >= T(0.5) ? 2 : 0);
                if (near == c) {
                    sum += oyv[2 * (int64_t)k];
                    ++cnt;
                }
            }
        }
    }
    __align__(16) __nv_bfloat16 o[16];
    o[0] = __float2bfloat16(cnt ? (float)(sum / T(cnt) * inv_scale) : 0.f);
    o[1] = __float2bfloat16(cnt ? 1.f : 0.f);
    o[2] = __float2bfloat16(kfeat);
#pragma unroll
    for (int c = 3; c < 16; ++c) o[c] = __float2bfloat16(0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(x + q * 16);
    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
}

// t[i][j] = (mu / scale, log Lambda) of the current beliefs (after k_beliefs); zeros in the pad
template <typename T> __global__ void k_ws_target(DevProblem p, double inv_scale, int Hp, int Wp, float *t) {
    const int64_t q = gtid();
    if (q >= (int64_t)Hp * Wp) return;
    int i, j;
    node_rc(q, Wp, i, j);
    float a = 0.f, b = 0.f;
    if (i < p.ny && j < p.nx) {
        const BeliefStore<T> s = ((const BeliefStore<T> *)p.belief)[(int64_t)i * p.nx + j];
        const double L = (double)s.lhi + (double)s.llo;
        a = (float)(((double)s.ehi + (double)s.elo) / L * inv_scale);
        b = (float)log(L);
    }
    t[2 * q] = a;
    t[2 * q + 1] = b;
}

// initial beliefs from the network output: mu0 = scale * out0, lam0 = exp(out1) clamped
// FP32 contexts: per node, the initial message pair (mu0 L, L) with L = lam0 / (number of factor
// slots at the node), decoded from the network output (mu0 = scale * out0, lam0 = exp(out1)
// with out1 clamped to [-10, 15]); the message planes are then gathered from it.
__global__ void k_ws_node_msg(DevProblem p, float scale, int Wp, const float *out, float2 *nm) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    const int64_t q = (int64_t)i * Wp + j;
    const float lg = fminf(fmaxf(out[2 * q + 1], -10.f), 15.f);
    const float L = expf(lg) / (float)node_slots(p, v);
    nm[v] = make_float2(scale * out[2 * q] * L, L);
}
// FP32 contexts: node message pairs from given marginals (mu0, lam0), as in the FP64 path but
// in FP32 arithmetic (L = lam0 / slots, eta = mu0 L)
__global__ void k_node_msg_marg(DevProblem p, const double *mu0, const double *lam0, float2 *nm) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    const float L = (float)lam0[v] / (float)node_slots(p, v);
    nm[v] = make_float2((float)mu0[v] * L, L);
}

// Multigrid upscaling (Alg. 2 "Upscale Messages", read as copying parent marginals): node (i, j)
// of the finer grid takes mean and precision of node (i >> shift, j >> shift) of the coarser
// (shift 1: the parent (floor(i/2), floor(j/2)); shift 0: the same grid, a plain copy);
// q_c holds variances (q_is_var) or precisions
__global__ void k_upscale_marg(const double *mu_c, const double *q_c, int q_is_var, int shift, int nxc, int nyc,
                               int nxf, int nyf, double *mu_f, double *lam_f) {
    const int64_t v = gtid();
    if (v >= (int64_t)nxf * nyf) return;
    int i, j;
    node_rc(v, nxf, i, j);
    const int ic = min(i >> shift, nyc - 1), jc = min(j >> shift, nxc - 1);
    const int64_t c = (int64_t)ic * nxc + jc;
    mu_f[v] = mu_c[c];
    lam_f[v] = q_is_var ? 1.0 / q_c[c] : q_c[c];
}

__global__ void k_init_nodes_prior(DevProblem p, int dst, const float2 *nm) {
    const int64_t c = gtid();
    if (c >= p.n) return;
    const int nx = p.nx, ny = p.ny;
    int i, j;
    node_rc(c, nx, i, j);
    const bool exists[5] = {true, j > 0, j < nx - 1, i > 0, i < ny - 1};
    const int64_t node[5] = {c, c - 1, c + 1, c - nx, c + nx};
    float2 *Q = (float2 *)p.P[dst];
#pragma unroll
    for (int u = 0; u < 5; ++u) Q[u * p.pn + plane_at(p, i, j)] = exists[u] ? nm[node[u]] : make_float2(0.f, 0.f);
}
__global__ void k_init_nodes_obs(DevProblem p, int dst, const float2 *nm) {
    const int64_t k = gtid();
    if (k >= p.m) return;
    const int64_t b = p.obase[k];
    const float2 m0 = nm[b], m1 = nm[b + 1], m2 = nm[b + p.nx], m3 = nm[b + p.nx + 1];
    float4 *Q = (float4 *)((float *)p.O[dst] + 8 * k);
    Q[0] = make_float4(m0.x, m0.y, m1.x, m1.y);
    Q[1] = make_float4(m2.x, m2.y, m3.x, m3.y);
}

__global__ void k_ws_decode(DevProblem p, double scale, int Wp, const float *out, double *mu0, double *lam0) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    const int64_t q = (int64_t)i * Wp + j;
    double lg = (double)out[2 * q + 1];
    lg = lg < -10.0 ? -10.0 : (lg > 15.0 ? 15.0 : lg);
    mu0[v] = scale * (double)out[2 * q];
    lam0[v] = exp(lg);
}

template <typename T> cudaError_t split_iteration(const DevProblem &p, int src, double beta, cudaStream_t st) {
    k_beliefs<T><<<nblocks(p.n), TPB, 0, st>>>(p, src);
    k_prior<T><<<nblocks(p.n), TPB, 0, st>>>(p, src, (T)beta);
    if (p.m > 0) k_obs<T><<<nblocks(p.m), TPB, 0, st>>>(p, src, (T)beta);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split_iteration(const DevProblem &p, int src, double beta, cudaStream_t st) {
    if (p.order == 2) return launch_l2_iteration(p, src, beta, st);
    return p.prec ? split_iteration<double>(p, src, beta, st) : split_iteration<float>(p, src, beta, st);
}

cudaError_t launch_l2_iteration(const DevProblem &p, int src, double beta, cudaStream_t st) {
    if (p.order != 2 || p.px != p.nx) return cudaErrorInvalidValue;   // alpha = 4 planes are unpadded
    if (p.prec) {
        k_beliefs_l2<double><<<row_grid(p.nx, p.ny), TPB, 0, st>>>(p, src);
        k_prior_l2<double><<<row_grid(p.nx, p.ny), TPB, 0, st>>>(p, src, beta);
        if (p.m > 0) k_obs<double><<<nblocks(p.m), TPB, 0, st>>>(p, src, beta);
    } else {
        k_beliefs_l2<float><<<row_grid(p.nx, p.ny), TPB, 0, st>>>(p, src);
        k_prior_l2<float><<<row_grid(p.nx, p.ny), TPB, 0, st>>>(p, src, (float)beta);
        if (p.m > 0) k_obs<float><<<nblocks(p.m), TPB, 0, st>>>(p, src, (float)beta);
    }
    return cudaGetLastError();
}

cudaError_t launch_beliefs(const DevProblem &p, int src, cudaStream_t st) {
    if (p.order == 2) {
        if (p.prec) k_beliefs_l2<double><<<row_grid(p.nx, p.ny), TPB, 0, st>>>(p, src);
        else k_beliefs_l2<float><<<row_grid(p.nx, p.ny), TPB, 0, st>>>(p, src);
        return cudaGetLastError();
    }
    if (p.prec) k_beliefs<double><<<nblocks(p.n), TPB, 0, st>>>(p, src);
    else k_beliefs<float><<<nblocks(p.n), TPB, 0, st>>>(p, src);
    return cudaGetLastError();
}

cudaError_t launch_init_cold(const DevProblem &p, int dst, int paper, cudaStream_t st) {
    if (p.order == 2) {
        if (p.prec) {
            k_init_prior_l2<double><<<nblocks(p.n), TPB, 0, st>>>(p, dst, paper);
            if (p.m > 0) k_init_obs<double><<<nblocks(p.m), TPB, 0, st>>>(p, dst, paper);
        } else {
            k_init_prior_l2<float><<<nblocks(p.n), TPB, 0, st>>>(p, dst, paper);
            if (p.m > 0) k_init_obs<float><<<nblocks(p.m), TPB, 0, st>>>(p, dst, paper);
        }
        return cudaGetLastError();
    }
    if (p.prec) {
        k_init_prior<double><<<nblocks(p.n), TPB, 0, st>>>(p, dst, paper);
        if (p.m > 0) k_init_obs<double><<<nblocks(p.m), TPB, 0, st>>>(p, dst, paper);
    } else {
        k_init_prior<float><<<nblocks(p.n), TPB, 0, st>>>(p, dst, paper);
        if (p.m > 0) k_init_obs<float><<<nblocks(p.m), TPB, 0, st>>>(p, dst, paper);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_warm(const DevProblem &p, int dst, const double *mu0, const double *lam0,
                             cudaStream_t st) {
    if (p.prec) {
        k_init_warm_prior<double><<<nblocks(p.n), TPB, 0, st>>>(p, dst, mu0, lam0);
        if (p.m > 0) k_init_warm_obs<double><<<nblocks(p.m), TPB, 0, st>>>(p, dst, mu0, lam0);
    } else {
        k_init_warm_prior<float><<<nblocks(p.n), TPB, 0, st>>>(p, dst, mu0, lam0);
        if (p.m > 0) k_init_warm_obs<float><<<nblocks(p.m), TPB, 0, st>>>(p, dst, mu0, lam0);
    }
    return cudaGetLastError();
}

cudaError_t launch_obs_precompute(const DevProblem &p, const double *xy, const double *yv,
                                  const double *var, cudaStream_t st) {
    if (p.m == 0) return cudaSuccess;
    if (p.prec) k_obs_precompute<double><<<nblocks(p.m), TPB, 0, st>>>(p, xy, yv, var);
    else k_obs_precompute<float><<<nblocks(p.m), TPB, 0, st>>>(p, xy, yv, var);
    return cudaGetLastError();
}

cudaError_t launch_obs_pointers(const DevProblem &p, cudaStream_t st) {
    k_obs_pointers<<<nblocks(p.n + 1), TPB, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_rhs_norm(const DevProblem &p, cudaStream_t st) {
    k_rhs_norm<<<RES_BLOCKS, TPB, 0, st>>>(p);
    k_final_sum<<<1, TPB, 0, st>>>(p.part, RES_BLOCKS, p.scal + 1);
    return cudaGetLastError();
}

// ---- message change between the last two iterates (the early-stopping rule of App. B) ----
// partial sums over a fixed grid of |m_t - m_{t-1}| for every stored message component: the
// prior planes (slots without a neighbour hold (0, 0) in both buffers and add nothing) and the
// observation messages.  Per-thread sums in T, block sums in FP64, fixed order.
template <typename T> __global__ void k_msg_change(DevProblem p, int cur) {
    const T *a = (const T *)p.P[cur], *b = (const T *)p.P[cur ^ 1];
    const T *oa = (const T *)p.O[cur], *ob = (const T *)p.O[cur ^ 1];
    const int64_t np_ = 2 * (int64_t)p.planes * p.pn, no = 8 * p.m;   // padding cells: (0, 0) in both
    const int64_t stride = (int64_t)gridDim.x * TPB;
    T acc = T(0);
    for (int64_t i = gtid(); i < np_; i += stride) acc += fabs(a[i] - b[i]);
    for (int64_t i = gtid(); i < no; i += stride) acc += fabs(oa[i] - ob[i]);
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) p.part[blockIdx.x] = s;
}

cudaError_t launch_msg_change(const DevProblem &p, int cur, double *out, cudaStream_t st) {
    if (p.prec) k_msg_change<double><<<RES_BLOCKS, TPB, 0, st>>>(p, cur);
    else k_msg_change<float><<<RES_BLOCKS, TPB, 0, st>>>(p, cur);
    k_final_sum<<<1, TPB, 0, st>>>(p.part, RES_BLOCKS, out);
    return cudaGetLastError();
}

cudaError_t launch_df_precompute(const DevProblem &p, cudaStream_t st) {
    if (p.m == 0 || p.prec) return cudaSuccess;
    k_df_precompute<<<nblocks(p.m), TPB, 0, st>>>(p);
    return cudaGetLastError();
}

// the residual of a mean already in p.mu64 (double-float pairs for FP32 contexts, FP64 values
// for FP64 contexts): the kernels after the mean in launch_residual
cudaError_t launch_residual_mu(const DevProblem &p, cudaStream_t st) {
    if (p.order == 2) return cudaErrorInvalidValue;   // order-2 contexts: launch_residual only
    if (p.prec == 0) {
        if (p.m > 0) k_obs_err_df<<<nblocks(p.m), TPB, 0, st>>>(p);
        k_Lmu_df<<<nblocks(p.n), TPB, 0, st>>>(p);
        k_res_df<<<RES_BLOCKS, TPB, 0, st>>>(p);
    } else {
        if (p.m > 0) k_obs_err<<<nblocks(p.m), TPB, 0, st>>>(p);
        k_Lmu<<<nblocks(p.n), TPB, 0, st>>>(p);
        k_res<<<RES_BLOCKS, TPB, 0, st>>>(p);
    }
    k_final_sum<<<1, TPB, 0, st>>>(p.part, RES_BLOCKS, p.scal);
    return cudaGetLastError();
}

cudaError_t launch_residual(const DevProblem &p, int src, cudaStream_t st) {
    if (p.order == 1 && p.prec == 0) {
        // FP32 messages: the residual in double-float arithmetic (FP32 pipes, ~48-bit significands)
        k_mu_direct_df<<<nblocks(p.n), TPB, 0, st>>>(p, src);
        if (p.m > 0) k_obs_err_df<<<nblocks(p.m), TPB, 0, st>>>(p);
        k_Lmu_df<<<nblocks(p.n), TPB, 0, st>>>(p);
        k_res_df<<<RES_BLOCKS, TPB, 0, st>>>(p);
        k_final_sum<<<1, TPB, 0, st>>>(p.part, RES_BLOCKS, p.scal);
        return cudaGetLastError();
    }
    cudaError_t e = launch_beliefs(p, src, st);
    if (e != cudaSuccess) return e;
    if (p.order == 2) {
        // r = b - gamma L^4 mu - H^T S (H mu - y) in FP64 (both precisions): z = L mu, then L
        // twice more through the scratch vectors, and k_res applies the fourth L
        if (p.prec) k_mu<double><<<nblocks(p.n), TPB, 0, st>>>(p);
        else k_mu<float><<<nblocks(p.n), TPB, 0, st>>>(p);
        if (p.m > 0) k_obs_err<<<nblocks(p.m), TPB, 0, st>>>(p);
        k_Lx<<<nblocks(p.n), TPB, 0, st>>>(p, p.mu64, p.z64);
        k_Lx<<<nblocks(p.n), TPB, 0, st>>>(p, p.z64, p.mu64);
        k_Lx<<<nblocks(p.n), TPB, 0, st>>>(p, p.mu64, p.z64);
        k_res<<<RES_BLOCKS, TPB, 0, st>>>(p);
        k_final_sum<<<1, TPB, 0, st>>>(p.part, RES_BLOCKS, p.scal);
        return cudaGetLastError();
    }
    if (p.prec) k_mu<double><<<nblocks(p.n), TPB, 0, st>>>(p);
    else k_mu<float><<<nblocks(p.n), TPB, 0, st>>>(p);
    if (p.m > 0) k_obs_err<<<nblocks(p.m), TPB, 0, st>>>(p);
    k_Lmu<<<nblocks(p.n), TPB, 0, st>>>(p);
    k_res<<<RES_BLOCKS, TPB, 0, st>>>(p);
    k_final_sum<<<1, TPB, 0, st>>>(p.part, RES_BLOCKS, p.scal);
    return cudaGetLastError();
}

cudaError_t launch_ws_input(const DevProblem &p, double scale, double kappa, int Hp, int Wp, void *x,
                            cudaStream_t st) {
    const float kf = (float)(std::log(kappa) + 3.0);
    if (p.prec)
        k_ws_input<double><<<nblocks((int64_t)Hp * Wp), TPB, 0, st>>>(p, 1.0 / scale, kf, Hp, Wp, (__nv_bfloat16 *)x);
    else
        k_ws_input<float><<<nblocks((int64_t)Hp * Wp), TPB, 0, st>>>(p, (float)(1.0 / scale), kf, Hp, Wp,
                                                                     (__nv_bfloat16 *)x);
    return cudaGetLastError();
}

cudaError_t launch_ws_target(const DevProblem &p, int src, double scale, int Hp, int Wp, float *t, cudaStream_t st) {
    cudaError_t e = launch_beliefs(p, src, st);
    if (e != cudaSuccess) return e;
    if (p.prec) k_ws_target<double><<<nblocks((int64_t)Hp * Wp), TPB, 0, st>>>(p, 1.0 / scale, Hp, Wp, t);
    else k_ws_target<float><<<nblocks((int64_t)Hp * Wp), TPB, 0, st>>>(p, 1.0 / scale, Hp, Wp, t);
    return cudaGetLastError();
}

cudaError_t launch_upscale(const double *mu_c, const double *q_c, int q_is_var, int shift, int nxc, int nyc, int nxf,
                           int nyf, double *mu_f, double *lam_f, cudaStream_t st) {
    k_upscale_marg<<<nblocks((int64_t)nxf * nyf), TPB, 0, st>>>(mu_c, q_c, q_is_var, shift, nxc, nyc, nxf, nyf, mu_f,
                                                                 lam_f);
    return cudaGetLastError();
}

cudaError_t launch_init_warm_f32(const DevProblem &p, int dst, const double *mu0, const double *lam0, float2 *nm,
                                 cudaStream_t st) {
    if (p.prec) return cudaErrorInvalidValue;
    k_node_msg_marg<<<nblocks(p.n), TPB, 0, st>>>(p, mu0, lam0, nm);
    k_init_nodes_prior<<<nblocks(p.n), TPB, 0, st>>>(p, dst, nm);
    if (p.m > 0) k_init_nodes_obs<<<nblocks(p.m), TPB, 0, st>>>(p, dst, nm);
    return cudaGetLastError();
}

cudaError_t launch_ws_init_f32(const DevProblem &p, int dst, double scale, int Wp, const float *out, float2 *nm,
                               cudaStream_t st) {
    if (p.prec) return cudaErrorInvalidValue;
    k_ws_node_msg<<<nblocks(p.n), TPB, 0, st>>>(p, (float)scale, Wp, out, nm);
    k_init_nodes_prior<<<nblocks(p.n), TPB, 0, st>>>(p, dst, nm);
    if (p.m > 0) k_init_nodes_obs<<<nblocks(p.m), TPB, 0, st>>>(p, dst, nm);
    return cudaGetLastError();
}

cudaError_t launch_ws_decode(const DevProblem &p, double scale, int Wp, const float *out, double *mu0, double *lam0,
                             cudaStream_t st) {
    k_ws_decode<<<nblocks(p.n), TPB, 0, st>>>(p, scale, Wp, out, mu0, lam0);
    return cudaGetLastError();
}

cudaError_t launch_marginals(const DevProblem &p, int src, double *mean, double *var, cudaStream_t st, bool direct) {
    if (p.order == 2 || !direct) {   // the beliefs first (13 planes; or outputs across the host link)
        cudaError_t e = launch_beliefs(p, src, st);
        if (e != cudaSuccess) return e;
        if (p.prec) k_marg_stored<double><<<nblocks(p.n), TPB, 0, st>>>(p, mean, var);
        else k_marg_stored<float><<<nblocks(p.n), TPB, 0, st>>>(p, mean, var);
        return cudaGetLastError();
    }
    if (p.prec) k_marg<double><<<nblocks(p.n), TPB, 0, st>>>(p, src, mean, var);
    else k_marg<float><<<nblocks(p.n), TPB, 0, st>>>(p, src, mean, var);
    return cudaGetLastError();
}


// ---- prior mean ----
// t = L d (FP64), rounded to the message precision and (FP32 contexts) split into double-float
template <typename T> __global__ void k_cell_targets(DevProblem p, const double *d, double *t64, T *tT, float2 *tdf) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    int i, j;
    node_rc(v, p.nx, i, j);
    const double t = d ? apply_L(p, d, v, i, j) : 0.0;
    t64[v] = t;
    tT[v] = (T)t;
    if (tdf) df_st(tdf, v, df_split(t));
}

cudaError_t launch_cell_targets(const DevProblem &p, const double *d, double *t64, void *tT, float2 *tdf,
                                cudaStream_t st) {
    if (p.prec == 0) k_cell_targets<float><<<nblocks(p.n), TPB, 0, st>>>(p, d, t64, (float *)tT, tdf);
    else k_cell_targets<double><<<nblocks(p.n), TPB, 0, st>>>(p, d, t64, (double *)tT, nullptr);
    return cudaGetLastError();
}

}  // namespace gabp
