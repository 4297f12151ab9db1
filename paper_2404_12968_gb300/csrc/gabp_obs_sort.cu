// Observation layout of context creation on the GPU: the base cell of every observation and a
// stable sort of the observations by base cell (ties keep their input order), the order every
// iteration kernel relies on, then the gather of the sorted raw data for the FP64 precompute.
//
// The sort is a least-significant-digit radix sort of (base cell, input index) pairs with 8-bit
// digits, ceil(log2 n) / 8 passes.  Each pass:
//   1. k_rs_hist: every block counts the digits of its chunk of 2048 pairs (shared-memory
//      counters: the counts are exact integers, so the result does not depend on timing);
//   2. an exclusive scan of the counts in (digit, block) order gives every (digit, block) its
//      first output position;
//   3. k_rs_scatter: every block walks its chunk in order, each warp a contiguous run of 256
//      pairs, 32 at a time; lanes holding the same digit find each other with a warp match and
//      take consecutive positions in lane order, after the pairs of the same digit in earlier
//      groups, warps and blocks.  So each pass is stable, and so is the sort.
// No step depends on the order in which blocks or atomics run.
#include <cstdint>

#include "gabp_internal.h"

namespace gabp {

namespace {

constexpr int RS_T = 256, RS_W = RS_T / 32, RS_PER_WARP = 256, RS_CHUNK = RS_W * RS_PER_WARP;
constexpr int RS_BITS = 8, RS_BINS = 1 << RS_BITS;
constexpr int SCAN_T = 256, SCAN_E = 8, SCAN_B = SCAN_T * SCAN_E;

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }

// base cell (FP64 floor of the location, clamped to the last full cell) and input index
__global__ void k_obs_keys(const double *xy, int64_t m, int nx, int ny, int *key, int *idx) {
    const int64_t k = gtid();
    if (k >= m) return;
    int j0 = (int)floor(xy[2 * k]), i0 = (int)floor(xy[2 * k + 1]);
    if (j0 > nx - 2) j0 = nx - 2;
    if (i0 > ny - 2) i0 = ny - 2;
    key[k] = i0 * nx + j0;
    idx[k] = (int)k;
}

__global__ void __launch_bounds__(RS_T) k_rs_hist(const int *key, int64_t m, int shift, int nblk, int *hist) {
    __shared__ int h[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += RS_T) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_CHUNK;
    for (int e = threadIdx.x; e < RS_CHUNK; e += RS_T) {
        const int64_t k = base + e;
        if (k < m) atomicAdd(&h[(key[k] >> shift) & (RS_BINS - 1)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RS_BINS; i += RS_T) hist[(int64_t)i * nblk + blockIdx.x] = h[i];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const int *key, const int *idx, int64_t m, int shift, int nblk,
                                                     const int *off, int *key2, int *idx2) {
    __shared__ int wc[RS_W][RS_BINS];   // per warp and digit: count, then next output position
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_W * RS_BINS; i += RS_T) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_CHUNK + warp * RS_PER_WARP;
    const unsigned lt = (1u << lane) - 1u;
    for (int g = 0; g < RS_PER_WARP; g += 32) {
        const int64_t k = wbase + g + lane;
        const bool valid = k < m;
        const int d = valid ? (key[k] >> shift) & (RS_BINS - 1) : RS_BINS;   // RS_BINS: no pair
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) wc[warp][d] += __popc(peers);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_T) {
        int run = off[(int64_t)d * nblk + blockIdx.x];
        for (int w = 0; w < RS_W; ++w) {
            const int t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int g = 0; g < RS_PER_WARP; g += 32) {
        const int64_t k = wbase + g + lane;
        const bool valid = k < m;
        const int kk = valid ? key[k] : 0;
        const int d = valid ? (kk >> shift) & (RS_BINS - 1) : RS_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid) {
            const int pos = wc[warp][d] + __popc(peers & lt);
            key2[pos] = kk;
            idx2[pos] = idx[k];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
}

// exclusive prefix sum of one value per thread over the block (SCAN_T threads)
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < SCAN_T / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < SCAN_T / 32) warp_tot[lane] = w;   // inclusive totals of the warps
    }
    __syncthreads();
    const int res = inc - v + (warp > 0 ? warp_tot[warp - 1] : 0);
    __syncthreads();
    return res;
}

// exclusive scan of in[0 .. count) into out, three phases: block sums, their scan, block scans
__global__ void __launch_bounds__(SCAN_T) k_scan_sums(const int *in, int64_t count, int *part) {
    __shared__ int wt[SCAN_T / 32];
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_B + threadIdx.x * SCAN_E;
    int s = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e)
        if (i0 + e < count) s += in[i0 + e];
    const int ex = block_exclusive_scan(s, wt);
    if (threadIdx.x == SCAN_T - 1) part[blockIdx.x] = ex + s;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_parts(int *part, int nparts) {
    __shared__ int wt[SCAN_T / 32];
    const int per = (nparts + SCAN_T - 1) / SCAN_T;
    const int lo = threadIdx.x * per, hi = min(lo + per, nparts);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += part[i];
    int run = block_exclusive_scan(s, wt);
    for (int i = lo; i < hi; ++i) {
        const int v = part[i];
        part[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const int *in, int64_t count, const int *part, int *out) {
    __shared__ int wt[SCAN_T / 32];
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_B + threadIdx.x * SCAN_E;
    int v[SCAN_E], s = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        v[e] = i0 + e < count ? in[i0 + e] : 0;
        s += v[e];
    }
    int run = block_exclusive_scan(s, wt) + part[blockIdx.x];
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        if (i0 + e < count) out[i0 + e] = run;
        run += v[e];
    }
}

__global__ void k_obs_gather(const int *key, const int *idx, int64_t m, const double *xy, const double *y,
                             const double *var, int *obase, double *sxy, double *sy, double *svar) {
    const int64_t d = gtid();
    if (d >= m) return;
    const int64_t k = idx[d];
    obase[d] = key[d];
    sxy[2 * d] = xy[2 * k];
    sxy[2 * d + 1] = xy[2 * k + 1];
    sy[d] = y[k];
    svar[d] = var[k];
}

inline unsigned blocks_for(int64_t count, int per) { return (unsigned)((count + per - 1) / per); }

}  // namespace

size_t obs_sort_scratch_bytes(int64_t m) {
    const int64_t nblk = (m + RS_CHUNK - 1) / RS_CHUNK;
    const int64_t hcount = (int64_t)RS_BINS * nblk;
    const int64_t nparts = (hcount + SCAN_B - 1) / SCAN_B;
    return sizeof(int) * (size_t)(4 * m + 2 * hcount + nparts + 64);
}

cudaError_t launch_obs_sort(int64_t m, int nx, int ny, const double *xy, const double *y, const double *var,
                            int *obase, double *sxy, double *sy, double *svar, void *scratch, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int64_t n = (int64_t)nx * ny;
    const int64_t nblk = (m + RS_CHUNK - 1) / RS_CHUNK;
    const int64_t hcount = (int64_t)RS_BINS * nblk;
    const int64_t nparts = (hcount + SCAN_B - 1) / SCAN_B;
    if (nparts > (int64_t)SCAN_T * 4096 || nblk > 0x7fffffff) return cudaErrorInvalidValue;
    int *key = static_cast<int *>(scratch), *idx = key + m, *key2 = idx + m, *idx2 = key2 + m;
    int *hist = idx2 + m, *off = hist + hcount, *part = off + hcount;
    k_obs_keys<<<blocks_for(m, 256), 256, 0, st>>>(xy, m, nx, ny, key, idx);
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
    for (int shift = 0; shift < bits; shift += RS_BITS) {
        k_rs_hist<<<(unsigned)nblk, RS_T, 0, st>>>(key, m, shift, (int)nblk, hist);
        k_scan_sums<<<(unsigned)nparts, SCAN_T, 0, st>>>(hist, hcount, part);
        k_scan_parts<<<1, SCAN_T, 0, st>>>(part, (int)nparts);
        k_scan_apply<<<(unsigned)nparts, SCAN_T, 0, st>>>(hist, hcount, part, off);
        k_rs_scatter<<<(unsigned)nblk, RS_T, 0, st>>>(key, idx, m, shift, (int)nblk, off, key2, idx2);
        int *t = key;
        key = key2;
        key2 = t;
        t = idx;
        idx = idx2;
        idx2 = t;
    }
    k_obs_gather<<<blocks_for(m, 256), 256, 0, st>>>(key, idx, m, xy, y, var, obase, sxy, sy, svar);
    return cudaGetLastError();
}

}  // namespace gabp
