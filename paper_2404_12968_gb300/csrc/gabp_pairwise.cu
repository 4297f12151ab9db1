// The paper's pairwise re-weighted Gaussian message passing (App. A, "Gaussian Setting" and
// "Re-weighted message updates"), as a second iteration family over the same posterior.
//
// Model: p(f) ~ exp(-f^T P f / 2 + h^T f) with P = gamma L^T L + H^T R^-1 H, h = H^T R^-1 y.
// One node factor per node and one pair factor per nonzero off-diagonal P_ij: the 13-point
// pattern of L^T L (offsets (0, +-1), (+-1, 0), (+-1, +-1), (0, +-2), (+-2, 0)); bilinear
// observations stay inside it.  Fractional messages with weight c (the information convention
// exp(-a f^2 / 2 + b f) throughout):
//   alpha_{j->i} = P_jj + c sum_{k != i} a_{kj} + (c - 1) a_{ij},
//   beta_{j->i}  = h_j  + c sum_{k != i} b_{kj} + (c - 1) b_{ij},
//   a_{ji} = -(P_ij / c)^2 / alpha_{j->i},   b_{ji} = -beta_{j->i} (P_ij / c) / alpha_{j->i},
// with (a_kj, b_kj) the pair factor (k, j)'s message to f_j.  The b update follows the integral
// that defines the message (the paper prints the opposite sign).  Damping with the paper's
// learning rate eta: m <- (1 - eta) m_old + eta m_new.  Marginal: mean (h_i + c sum_k b_ki) /
// (P_ii + c sum_k a_ki), precision P_ii + c sum_k a_ki.
//
// Layout: 12 "outgoing" planes of (a, b) pairs, ping-pong: plane d at node j holds the message of
// the pair factor (j, j + off_d) to f_{j + off_d}, computed by node j; slots without that
// neighbour hold (0, 0).  Node i reads its incoming messages from plane d at i - off_d, and
// the pair factor's message back to itself from plane opp(d) at i + off_d.  Coefficients per
// node: P_ii, h_i and P_{i, i + off_d}.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "gabp_device.cuh"
#include "gabp_internal.h"

namespace gabp {

namespace {

constexpr int PW_TPB = 256;
constexpr int ND = 12;
// (dy, dx) of the 12 directions, ordered so that the opposite of direction d is d ^ 1; the
// first 8 are the nearest offsets (every corner pair of an observation cell)
__host__ __device__ constexpr int DY(int d) {
    return d == 2 || d == 4 || d == 6 ? -1 : d == 3 || d == 5 || d == 7 ? 1 : d == 10 ? -2 : d == 11 ? 2 : 0;
}
__host__ __device__ constexpr int DX(int d) {
    return d == 0 || d == 4 || d == 7 ? -1 : d == 1 || d == 5 || d == 6 ? 1 : d == 8 ? -2 : d == 9 ? 2 : 0;
}
__host__ __device__ constexpr int OPP(int d) { return d ^ 1; }

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
inline unsigned nblk(int64_t count) { return (unsigned)((count + PW_TPB - 1) / PW_TPB); }

// coefficient of node v in row c of L (zero-Neumann): kappa^2 + deg(c) on the diagonal, -1 for an
// existing 4-neighbour, 0 otherwise
__device__ __forceinline__ double L_coef(const DevProblem &p, int ci, int cj, int vi, int vj) {
    if (ci < 0 || ci >= p.ny || cj < 0 || cj >= p.nx) return 0.0;
    if (vi == ci && vj == cj) return p.aC[grid_degree(ci, cj, p.nx, p.ny)];
    const int d = abs(vi - ci) + abs(vj - cj);
    return d == 1 ? -1.0 : 0.0;
}

// Per node i: P_ii, h_i and P_{i, i + off_d} (FP64 sums, stored in T).  Prior: gamma sum over the
// cells c of the two nodes' stencils of L_ci L_cj; observations: s_k w_a w_b and s_k y_k w_a over
// the observations based in the four cells around i, in the order of the observation index.
template <typename T>
__global__ void k_pw_coef(DevProblem p, T *Pd, T *hv, T *Pn) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    const int nx = p.nx, ny = p.ny;
    const int i = (int)(v / nx), j = (int)(v - (int64_t)i * nx);
    double diag = 0.0, off[ND];
    for (int d = 0; d < ND; ++d) off[d] = 0.0;
    // prior: cells c in {v} and its 4-neighbours
    const int cdy[5] = {0, 0, 0, -1, 1}, cdx[5] = {0, -1, 1, 0, 0};
    for (int q = 0; q < 5; ++q) {
        const int ci = i + cdy[q], cj = j + cdx[q];
        const double li = L_coef(p, ci, cj, i, j);
        if (li == 0.0) continue;
        diag += p.gamma * li * li;
        for (int d = 0; d < ND; ++d) {
            const int ti = i + DY(d), tj = j + DX(d);
            if (ti < 0 || ti >= ny || tj < 0 || tj >= nx) continue;
            off[d] += p.gamma * li * L_coef(p, ci, cj, ti, tj);
        }
    }
    // observations based in the cells (i, j), (i, j-1), (i-1, j), (i-1, j-1): node v is corner
    // 0, 1, 2, 3 of them respectively; corner c sits at (dy, dx) = (c >> 1, c & 1) from the base
    double hh = 0.0;
    if (p.m > 0) {
        const int *o = p.optr;
        for (int cc = 0; cc < 4; ++cc) {
            const int bi = i - (cc >> 1), bj = j - (cc & 1);
            if (bi < 0 || bj < 0 || bi > ny - 2 || bj > nx - 2) continue;
            const int64_t b = (int64_t)bi * nx + bj;
            for (int k = o[b]; k < o[b + 1]; ++k) {
                const double *w = p.ow64 + 4 * (int64_t)k;
                const double s = p.oys64[2 * (int64_t)k + 1], y = p.oys64[2 * (int64_t)k];
                diag += s * w[cc] * w[cc];
                hh += s * y * w[cc];
                for (int c2 = 0; c2 < 4; ++c2) {
                    if (c2 == cc) continue;
                    const int ddy = (c2 >> 1) - (cc >> 1), ddx = (c2 & 1) - (cc & 1);
                    for (int d = 0; d < 8; ++d)   // the 8 nearest offsets hold every corner pair
                        if (DY(d) == ddy && DX(d) == ddx) off[d] += s * w[cc] * w[c2];
                }
            }
        }
    }
    Pd[v] = T(diag);
    hv[v] = T(hh);
    for (int d = 0; d < ND; ++d) Pn[(int64_t)d * p.n + v] = T(off[d]);
}

template <typename T>
__global__ void k_pw_zero(T *m, int64_t count) {
    const int64_t q = gtid();
    if (q < count) m[q] = T(0);
}

// One node's update (INTERIOR: all 12 neighbours exist, no bounds tests).  FP32: 1 / c is
// passed in (q = P_ij * (1 / c)) and 1 / alpha is the approximate reciprocal (as in the rank-1
// kernels); FP64: IEEE divisions.
template <typename T, bool INTERIOR>
__device__ __forceinline__ void pw_node(const DevProblem &p, int64_t v, int i, int j, const T *Pd, const T *hv,
                                        const T *Pn, const T2<T> *src, T2<T> *dst, T c, T inv_c, T eta) {
    const int nx = p.nx, ny = p.ny;
    const int64_t n = p.n;
    bool ex[ND];
    T ina[ND], inb[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const int ti = i + DY(d), tj = j + DX(d);
        ex[d] = INTERIOR || (ti >= 0 && ti < ny && tj >= 0 && tj < nx);
        // incoming from the neighbour at -off_d: plane d there
        const int si = i - DY(d), sj = j - DX(d);
        T2<T> m;
        m.x = T(0);
        m.y = T(0);
        if (INTERIOR || (si >= 0 && si < ny && sj >= 0 && sj < nx))
            m = src[(int64_t)d * n + v - ((int64_t)DY(d) * nx + DX(d))];
        ina[d] = m.x;
        inb[d] = m.y;
    }
    // leave-one-out sums of the incoming messages, in direction order
    T pa[ND + 1], pb[ND + 1];
    pa[0] = T(0);
    pb[0] = T(0);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        pa[d + 1] = add_rn(pa[d], ina[d]);
        pb[d + 1] = add_rn(pb[d], inb[d]);
    }
    T sa[ND + 1], sb[ND + 1];
    sa[ND] = T(0);
    sb[ND] = T(0);
#pragma unroll
    for (int d = ND - 1; d >= 0; --d) {
        sa[d] = add_rn(sa[d + 1], ina[d]);
        sb[d] = add_rn(sb[d + 1], inb[d]);
    }
    const T pjj = Pd[v], hj = hv[v], cm1 = add_rn(c, T(-1)), keep = add_rn(T(1), -eta);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        T2<T> out;
        out.x = T(0);
        out.y = T(0);
        if (ex[d]) {
            // the message of pair (j, i = j + off_d) back to f_j arrives from direction opp(d)
            const int r = OPP(d);
            const T loo_a = add_rn(pa[r], sa[r + 1]), loo_b = add_rn(pb[r], sb[r + 1]);
            const T alpha = add_rn(add_rn(pjj, mul_rn(c, loo_a)), mul_rn(cm1, ina[r]));
            const T beta = add_rn(add_rn(hj, mul_rn(c, loo_b)), mul_rn(cm1, inb[r]));
            T q, ra;
            if constexpr (sizeof(T) == 4) {
                q = mul_rn(Pn[(int64_t)d * n + v], inv_c);
                ra = recip(alpha);
            } else {
                q = Pn[(int64_t)d * n + v] / c;
                ra = T(1) / alpha;
            }
            const T an = -mul_rn(mul_rn(q, q), ra), bn = -mul_rn(mul_rn(beta, q), ra);
            const T2<T> old = src[(int64_t)d * n + v];
            // (1 - eta) old + eta new, as new + (1 - eta)(old - new)
            out.x = fma_rn(keep, add_rn(old.x, -an), an);
            out.y = fma_rn(keep, add_rn(old.y, -bn), bn);
        }
        __stcs(reinterpret_cast<T2<T> *>(dst) + (int64_t)d * n + v, out);
    }
}

// One synchronous iteration: node j reads its 12 incoming messages, forms the leave-one-out sums
// by prefix and suffix sums, and writes its 12 outgoing messages (damped).  FP32: registers
// bounded for 6 resident blocks of 256 threads per SM; the spills land in L1 and the extra
// loads in flight outweigh them (0.89 ms against 1.14 ms at 3 blocks, 4096^2).
template <typename T>
__global__ void __launch_bounds__(PW_TPB, sizeof(T) == 4 ? 6 : 1) k_pw_iter(DevProblem p, const T *Pd, const T *hv, const T *Pn, const T2<T> *src, T2<T> *dst, T c,
                          T inv_c, T eta) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    const int nx = p.nx, ny = p.ny;
    const int i = (int)(v / nx), j = (int)(v - (int64_t)i * nx);
    if (i >= 2 && i < ny - 2 && j >= 2 && j < nx - 2) pw_node<T, true>(p, v, i, j, Pd, hv, Pn, src, dst, c, inv_c, eta);
    else pw_node<T, false>(p, v, i, j, Pd, hv, Pn, src, dst, c, inv_c, eta);
}

// marginals (mean, precision) into mean / var arrays (FP64) or the residual's mean slot
template <typename T>
__global__ void k_pw_marg(DevProblem p, const T *Pd, const T *hv, const T2<T> *msg, T c, double *mean, double *var,
                          int to_residual) {
    const int64_t v = gtid();
    if (v >= p.n) return;
    const int nx = p.nx, ny = p.ny;
    const int64_t n = p.n;
    const int i = (int)(v / nx), j = (int)(v - (int64_t)i * nx);
    double sa = 0.0, sb = 0.0;
    for (int d = 0; d < ND; ++d) {
        const int si = i - DY(d), sj = j - DX(d);
        if (si < 0 || si >= ny || sj < 0 || sj >= nx) continue;
        const T2<T> m = msg[(int64_t)d * n + (int64_t)si * nx + sj];
        sa += (double)m.x;
        sb += (double)m.y;
    }
    const double prec = (double)Pd[v] + (double)c * sa;
    const double mu = ((double)hv[v] + (double)c * sb) / prec;
    if (to_residual) {
        if (p.prec == 0) {   // double-float pair for the FP32 contexts' residual kernels
            const float hi = __double2float_rn(mu);
            ((float2 *)p.mu64)[v] = make_float2(hi, __double2float_rn(mu - (double)hi));
        } else {
            p.mu64[v] = mu;
        }
    } else {
        mean[v] = mu;
        if (var) var[v] = 1.0 / prec;
    }
}

}  // namespace

cudaError_t pw_setup(const DevProblem &p, void *Pd, void *hv, void *Pn, cudaStream_t st) {
    if (p.prec) k_pw_coef<double><<<nblk(p.n), PW_TPB, 0, st>>>(p, (double *)Pd, (double *)hv, (double *)Pn);
    else k_pw_coef<float><<<nblk(p.n), PW_TPB, 0, st>>>(p, (float *)Pd, (float *)hv, (float *)Pn);
    return cudaGetLastError();
}

cudaError_t pw_zero(const DevProblem &p, void *msg, cudaStream_t st) {
    const int64_t count = 2 * ND * p.n;
    if (p.prec) k_pw_zero<double><<<nblk(count), PW_TPB, 0, st>>>((double *)msg, count);
    else k_pw_zero<float><<<nblk(count), PW_TPB, 0, st>>>((float *)msg, count);
    return cudaGetLastError();
}

cudaError_t pw_iterate(const DevProblem &p, const void *Pd, const void *hv, const void *Pn, const void *src, void *dst,
                       double c, double eta, cudaStream_t st) {
    if (p.prec)
        k_pw_iter<double><<<nblk(p.n), PW_TPB, 0, st>>>(p, (const double *)Pd, (const double *)hv, (const double *)Pn,
                                                        (const double2 *)src, (double2 *)dst, c, 1.0 / c, eta);
    else
        k_pw_iter<float><<<nblk(p.n), PW_TPB, 0, st>>>(p, (const float *)Pd, (const float *)hv, (const float *)Pn,
                                                       (const float2 *)src, (float2 *)dst, (float)c,
                                                       (float)(1.0 / c), (float)eta);
    return cudaGetLastError();
}

namespace {

// ---- Alg. 2 around the pairwise form: early stopping and upscaling ----

// Partial sums of |m_new - m_old| over both components of every stored message (slots without
// a neighbour hold (0, 0) in both buffers and add nothing), per-thread sums in T, block sums in
// FP64 in a fixed order; part[blockIdx.x] receives the block's sum.
template <typename T> __global__ void k_pw_change(int64_t count, const T *a, const T *b, double *part) {
    __shared__ double sh[PW_TPB];
    T acc = T(0);
    for (int64_t i = gtid(); i < count; i += (int64_t)gridDim.x * PW_TPB) acc += fabs(a[i] - b[i]);
    sh[threadIdx.x] = (double)acc;
    __syncthreads();
    for (int s2 = PW_TPB / 2; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) sh[threadIdx.x] += sh[threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_pw_sum(const double *part, int count, double *out) {
    __shared__ double sh[PW_TPB];
    double acc = 0.0;
    for (int q = threadIdx.x; q < count; q += PW_TPB) acc += part[q];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s2 = PW_TPB / 2; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) sh[threadIdx.x] += sh[threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// "Upscale Messages": fine plane d at node v = coarse plane d at v's parent (floor(i/2),
// floor(j/2)) when the fine node has that neighbour and the parent has it too, else (0, 0).
template <typename T>
__global__ void k_pw_upscale(int nxc, int nyc, int nxf, int nyf, const T2<T> *coarse, T2<T> *fine) {
    const int64_t v = gtid();
    const int64_t nf = (int64_t)nxf * nyf, nc = (int64_t)nxc * nyc;
    if (v >= nf) return;
    const int i = (int)(v / nxf), j = (int)(v - (int64_t)i * nxf);
    const int pi = min(i / 2, nyc - 1), pj = min(j / 2, nxc - 1);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        T2<T> m;
        m.x = T(0);
        m.y = T(0);
        const int ti = i + DY(d), tj = j + DX(d), ci = pi + DY(d), cj = pj + DX(d);
        if (ti >= 0 && ti < nyf && tj >= 0 && tj < nxf && ci >= 0 && ci < nyc && cj >= 0 && cj < nxc)
            m = coarse[(int64_t)d * nc + (int64_t)pi * nxc + pj];
        fine[(int64_t)d * nf + v] = m;
    }
}

}  // namespace

// directed edges of the pairwise form on an nx x ny grid (pairs within the 12 offsets)
int64_t pw_edge_count(int nx, int ny) {
    int64_t e = 0;
    for (int d = 0; d < ND; ++d) e += (int64_t)std::max(0, nx - std::abs(DX(d))) * std::max(0, ny - std::abs(DY(d)));
    return e;
}

cudaError_t pw_change(const DevProblem &p, const void *a, const void *b, double *part, int nparts, double *out,
                      cudaStream_t st) {
    const int64_t count = 2 * (int64_t)ND * p.n;
    if (p.prec) k_pw_change<double><<<nparts, PW_TPB, 0, st>>>(count, (const double *)a, (const double *)b, part);
    else k_pw_change<float><<<nparts, PW_TPB, 0, st>>>(count, (const float *)a, (const float *)b, part);
    k_pw_sum<<<1, PW_TPB, 0, st>>>(part, nparts, out);
    return cudaGetLastError();
}

cudaError_t pw_upscale(const DevProblem &fine, const DevProblem &coarse, const void *coarse_msg, void *fine_msg,
                       cudaStream_t st) {
    if (fine.prec != coarse.prec) return cudaErrorInvalidValue;
    if (fine.prec)
        k_pw_upscale<double><<<nblk(fine.n), PW_TPB, 0, st>>>(coarse.nx, coarse.ny, fine.nx, fine.ny,
                                                              (const double2 *)coarse_msg, (double2 *)fine_msg);
    else
        k_pw_upscale<float><<<nblk(fine.n), PW_TPB, 0, st>>>(coarse.nx, coarse.ny, fine.nx, fine.ny,
                                                             (const float2 *)coarse_msg, (float2 *)fine_msg);
    return cudaGetLastError();
}

cudaError_t pw_marginals(const DevProblem &p, const void *Pd, const void *hv, const void *msg, double c, double *mean,
                         double *var, int to_residual, cudaStream_t st) {
    if (p.prec)
        k_pw_marg<double><<<nblk(p.n), PW_TPB, 0, st>>>(p, (const double *)Pd, (const double *)hv, (const double2 *)msg,
                                                        c, mean, var, to_residual);
    else
        k_pw_marg<float><<<nblk(p.n), PW_TPB, 0, st>>>(p, (const float *)Pd, (const float *)hv, (const float2 *)msg,
                                                       (float)c, mean, var, to_residual);
    return cudaGetLastError();
}

}  // namespace gabp
