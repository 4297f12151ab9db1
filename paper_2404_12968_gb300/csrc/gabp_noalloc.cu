// gabp_residual_noalloc: the relative residual ||b - A mu|| / ||b|| of a caller-supplied mean,
// computed without allocating any device or host memory.
//
// Who needs it: callers that must not or cannot call cudaMalloc themselves or through this
// library, e.g. a process whose device memory is already held by another allocator (a deep
// learning framework's caching allocator keeps freed blocks, so a plain cudaMalloc can fail
// while the framework still has room) or a service loop with a fixed memory budget checked at
// start-up.  They pass every input and the output in memory they already own.
//
// Scratch: the file-scope device array `g_noalloc_scratch` (GABP_NOALLOC_MAX_DOUBLES doubles,
// 24 MiB), present on every GPU that loads the library until the process exits.  It holds
// (L mu) per node, the weighted observation residual per observation, the block partial sums
// and a validity flag.  Every call shares it and it keeps the last call's contents; the flag
// is cleared at the start of each call and every other word is written before it is read.
// Calls that overlap on the GPU (two streams, or two host threads) race on it.
//
// The kernels mirror the library's residual (gabp_split.cu): same stencil, same observation
// weights, same fixed reduction partition, corners summed in the same order.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "gabp.h"
#include "gabp_device.cuh"
#include "gabp_internal.h"

namespace {

static __device__ __align__(256) double g_noalloc_scratch[GABP_NOALLOC_MAX_DOUBLES];

constexpr int NA_TPB = 256;
constexpr int NA_BLOCKS = gabp::RES_BLOCKS;   // the residual's reduction partition

struct NaArgs {
    int nx, ny;
    int64_t n, m;
    double gamma;
    double aC[5];
    const double *xy, *y, *var, *mu;
    double *z, *e, *part;
    int *flag;
};

__device__ __forceinline__ int64_t na_tid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }

// base cell of observation k (FP64 floor, clamped into the last cell), as gabp_create does
__device__ __forceinline__ int64_t na_base(const NaArgs &a, int64_t k) {
    int j0 = (int)floor(a.xy[2 * k]), i0 = (int)floor(a.xy[2 * k + 1]);
    if (j0 > a.nx - 2) j0 = a.nx - 2;
    if (i0 > a.ny - 2) i0 = a.ny - 2;
    return (int64_t)i0 * a.nx + j0;
}

__device__ __forceinline__ double na_L(const NaArgs &a, const double *x, int64_t v, int i, int j) {
    double s = a.aC[gabp::grid_degree(i, j, a.nx, a.ny)] * x[v];
    if (j > 0) s -= x[v - 1];
    if (j < a.nx - 1) s -= x[v + 1];
    if (i > 0) s -= x[v - a.nx];
    if (i < a.ny - 1) s -= x[v + a.nx];
    return s;
}

__global__ void na_Lmu(NaArgs a) {
    const int64_t v = na_tid();
    if (v >= a.n) return;
    const int i = (int)(v / a.nx), j = (int)(v - (int64_t)i * a.nx);
    a.z[v] = na_L(a, a.mu, v, i, j);
}

// bilinear weights of observation k at its base cell
__device__ __forceinline__ void na_weights(const NaArgs &a, int64_t k, int64_t b, double w[4]) {
    const int i0 = (int)(b / a.nx), j0 = (int)(b - (int64_t)i0 * a.nx);
    const double fu = a.xy[2 * k] - (double)j0, fv = a.xy[2 * k + 1] - (double)i0;
    w[0] = (1.0 - fu) * (1.0 - fv);
    w[1] = fu * (1.0 - fv);
    w[2] = (1.0 - fu) * fv;
    w[3] = fu * fv;
}

// e_k = (H mu - y)_k / sigma_k^2; flags unsorted or out-of-grid observations
__global__ void na_obs(NaArgs a) {
    const int64_t k = na_tid();
    if (k >= a.m) return;
    const double x = a.xy[2 * k], yy = a.xy[2 * k + 1];
    if (!(x >= 0.0 && x <= a.nx - 1.0 && yy >= 0.0 && yy <= a.ny - 1.0) || !(a.var[k] > 0.0)) {
        atomicMax(a.flag, 2);   // takes precedence over "unsorted"
        a.e[k] = 0.0;
        return;
    }
    const int64_t b = na_base(a, k);
    if (k > 0 && na_base(a, k - 1) > b) atomicMax(a.flag, 1);
    double w[4];
    na_weights(a, k, b, w);
    const double hm = w[0] * a.mu[b] + w[1] * a.mu[b + 1] + w[2] * a.mu[b + a.nx] + w[3] * a.mu[b + a.nx + 1];
    a.e[k] = (1.0 / a.var[k]) * (hm - a.y[k]);
}

// first observation whose base cell is >= c (observations sorted by base cell)
__device__ __forceinline__ int64_t na_lower(const NaArgs &a, int64_t c) {
    int64_t lo = 0, hi = a.m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (na_base(a, mid) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double na_block_sum(double x) {
    __shared__ double sh[NA_TPB];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int s = NA_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// per node: r_v = -gamma (L z)_v - sum of w e over incident observations, b_v = sum of w s y;
// block partial sums of r^2 and b^2
__global__ void na_res(NaArgs a) {
    double ar = 0.0, ab = 0.0;
    const int64_t stride = (int64_t)gridDim.x * NA_TPB;
    for (int64_t v = na_tid(); v < a.n; v += stride) {
        const int i = (int)(v / a.nx), j = (int)(v - (int64_t)i * a.nx);
        double r = -a.gamma * na_L(a, a.z, v, i, j);
        double bv = 0.0;
        if (a.m > 0) {
            // corners 0..3: base cells v, v-1, v-nx, v-nx-1
            const int64_t bases[4] = {v, v - 1, v - a.nx, v - a.nx - 1};
            const bool ok[4] = {true, j > 0, i > 0, i > 0 && j > 0};
            double acc = 0.0;
            for (int c = 0; c < 4; ++c) {
                if (!ok[c]) continue;
                const int64_t k0 = na_lower(a, bases[c]), k1 = na_lower(a, bases[c] + 1);
                for (int64_t k = k0; k < k1; ++k) {
                    double w[4];
                    na_weights(a, k, bases[c], w);
                    acc += w[c] * a.e[k];
                    bv += w[c] * a.y[k] * (1.0 / a.var[k]);
                }
            }
            r -= acc;
        }
        ar += r * r;
        ab += bv * bv;
    }
    const double sr = na_block_sum(ar);
    const double sb = na_block_sum(ab);
    if (threadIdx.x == 0) {
        a.part[2 * blockIdx.x] = sr;
        a.part[2 * blockIdx.x + 1] = sb;
    }
}

__global__ void na_final(NaArgs a) {
    double ar = 0.0, ab = 0.0;
    for (int q = threadIdx.x; q < NA_BLOCKS; q += NA_TPB) {
        ar += a.part[2 * q];
        ab += a.part[2 * q + 1];
    }
    const double sr = na_block_sum(ar);
    const double sb = na_block_sum(ab);
    if (threadIdx.x == 0) {
        a.part[2 * NA_BLOCKS] = sr;
        a.part[2 * NA_BLOCKS + 1] = sb;
    }
}

// Address of the scratch array on each device, looked up once per device (with that device
// current) on the first call there.
constexpr int NA_MAX_DEV = 64;
std::once_flag g_once[NA_MAX_DEV];
double *g_addr[NA_MAX_DEV];
cudaError_t g_addr_err[NA_MAX_DEV];

thread_local char g_msg[256];

int na_fail(int code, const char *msg) {
    std::snprintf(g_msg, sizeof g_msg, "%s", msg);
    return code;
}

}  // namespace

extern "C" const char *gabp_residual_noalloc_error(void) { return g_msg; }

extern "C" int gabp_residual_noalloc(gabp_grid grid, double kappa, double gamma, int64_t m,
                                     const double *obs_xy, const double *y, const double *noise_var,
                                     const double *mean, double *rel_residual, void *stream) {
    g_msg[0] = 0;
    if (!rel_residual || !mean) return na_fail(GABP_ERR_ARG, "mean and rel_residual must not be NULL");
    if (grid.nx < 1 || grid.ny < 1 || !(grid.h == 1.0)) return na_fail(GABP_ERR_ARG, "bad grid");
    if (!(kappa > 0.0) || !std::isfinite(kappa) || !(gamma > 0.0) || !std::isfinite(gamma))
        return na_fail(GABP_ERR_ARG, "kappa and gamma must be finite and > 0");
    if (m < 0) return na_fail(GABP_ERR_ARG, "negative observation count");
    if (m > 0 && (!obs_xy || !y || !noise_var)) return na_fail(GABP_ERR_ARG, "observation arrays must not be NULL");
    if (m > 0 && (grid.nx < 2 || grid.ny < 2)) return na_fail(GABP_ERR_ARG, "observations need a grid of at least 2 x 2");
    const int64_t n = (int64_t)grid.nx * grid.ny;
    const int64_t need = n + m + 2 * (int64_t)NA_BLOCKS + 4;
    if (need > (int64_t)GABP_NOALLOC_MAX_DOUBLES) {
        std::snprintf(g_msg, sizeof g_msg,
                      "problem too large for the static scratch: n + m = %lld exceeds %lld",
                      (long long)(n + m), (long long)(GABP_NOALLOC_MAX_DOUBLES - 2 * NA_BLOCKS - 4));
        return GABP_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEV) {
        cudaGetLastError();
        return na_fail(GABP_ERR_CUDA, "no usable current CUDA device");
    }
    std::call_once(g_once[dev], [dev] {
        g_addr_err[dev] = cudaGetSymbolAddress((void **)&g_addr[dev], g_noalloc_scratch);
    });
    if (g_addr_err[dev] != cudaSuccess) return na_fail(GABP_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    double *scratch = g_addr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    // every array the kernels read must be device (or managed) memory of this device
    const void *ins[4] = {mean, obs_xy, y, noise_var};
    for (int q = 0; q < (m > 0 ? 4 : 1); ++q) {
        cudaPointerAttributes pa;
        e = cudaPointerGetAttributes(&pa, ins[q]);
        if (e != cudaSuccess || !(pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) ||
            (pa.type == cudaMemoryTypeDevice && pa.device != dev)) {
            cudaGetLastError();
            return na_fail(GABP_ERR_ARG, "inputs must be device memory of the current device");
        }
    }

    NaArgs a;
    a.nx = grid.nx;
    a.ny = grid.ny;
    a.n = n;
    a.m = m;
    a.gamma = gamma;
    for (int d = 0; d <= 4; ++d) a.aC[d] = kappa * kappa + (double)d;
    a.xy = obs_xy;
    a.y = y;
    a.var = noise_var;
    a.mu = mean;
    a.z = scratch;
    a.e = scratch + n;
    a.part = scratch + n + m;
    a.flag = reinterpret_cast<int *>(scratch + n + m + 2 * NA_BLOCKS + 2);

    e = cudaMemsetAsync(a.flag, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        na_Lmu<<<(unsigned)((n + NA_TPB - 1) / NA_TPB), NA_TPB, 0, st>>>(a);
        if (m > 0) na_obs<<<(unsigned)((m + NA_TPB - 1) / NA_TPB), NA_TPB, 0, st>>>(a);
        na_res<<<NA_BLOCKS, NA_TPB, 0, st>>>(a);
        na_final<<<1, NA_TPB, 0, st>>>(a);
        e = cudaGetLastError();
    }
    double sums[2] = {0.0, 0.0};
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums, a.part + 2 * NA_BLOCKS, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, a.flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::snprintf(g_msg, sizeof g_msg, "CUDA error: %s", cudaGetErrorString(e));
        return GABP_ERR_CUDA;
    }
    if (flag == 2) return na_fail(GABP_ERR_ARG, "an observation lies outside the grid or has a non-positive variance");
    if (flag == 1) return na_fail(GABP_ERR_ARG, "observations must be sorted by base cell");
    *rel_residual = sums[1] > 0.0 ? std::sqrt(sums[0]) / std::sqrt(sums[1]) : std::sqrt(sums[0]);
    return GABP_OK;
}
