// Fused GaBP iteration, FP32, as a warp-synchronous column sweep.
//
// Work unit: a strip of 30 columns x H rows owned by one warp.  Lane l covers column
// x0 - 1 + l: lanes 1..30 own the strip's cells, lanes 0 and 31 are a one-column halo whose
// beliefs the edge cells need.  The warp walks its rows top to bottom keeping, in registers,
//   * the 5 outgoing messages (C, W, E, S, N) of rows r, r+1, r+2 and a prefetch of row r+3,
//   * the compensated beliefs of rows r-1, r, r+1, and the observation index of rows r, r+1;
// the x-neighbours come from warp shuffles.  At row r it forms the belief of row r+1, then
// updates the cell factors of row r and the observation factors based in row r, and writes
// the damped messages to the other ping-pong buffer.  Every message is loaded from HBM once
// (coalesced 256-byte row segments), no shared memory and no block barrier is used, and the
// only recomputation is the one-column halo (1/16 of the beliefs) and two extra belief rows per
// strip.  The arithmetic and the summation order are those of the other iteration kernels, so
// the messages are bit-identical to theirs.
#include "gabp_device.cuh"
#include "gabp_internal.h"

namespace gabp {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SW = 30;   // owned columns per warp

struct Row5 {
    float2 m[5];   // C, W, E, S, N
};

// planes: node (x, y) of plane d at d * pn + y * px + x (px >= nx: the padded row pitch)
__device__ __forceinline__ Row5 load_row(const float2 *P, int64_t pn, int px, int nx, int ny, int x, int y) {
    Row5 r;
    if (x >= 0 && x < nx && y >= 0 && y < ny) {
        const int64_t c = (int64_t)y * px + x;
#pragma unroll
        for (int d = 0; d < 5; ++d) r.m[d] = __ldg(P + d * pn + c);
    } else {
#pragma unroll
        for (int d = 0; d < 5; ++d) r.m[d] = make_float2(0.f, 0.f);
    }
    return r;
}

__device__ __forceinline__ float2 load_one(const float2 *P, int64_t pn, int px, int nx, int ny, int d, int x, int y) {
    if (x >= 0 && x < nx && y >= 0 && y < ny) return __ldg(P + d * pn + (int64_t)y * px + x);
    return make_float2(0.f, 0.f);
}

__device__ __forceinline__ int load_optr(const int *optr, int nx, int ny, int x, int y) {
    // observations with base cell before (x, y); 0 outside the grid (only used for in-grid
    // ranges: the callers test the column and row of the base cell first)
    if (x >= 0 && x < nx && y >= 0 && y < ny) return __ldg(optr + (int64_t)y * nx + x);
    return 0;
}

__device__ __forceinline__ float2 shfl_up2(float2 v) {
    return make_float2(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down2(float2 v) {
    return make_float2(__shfl_down_sync(FULL, v.x, 1), __shfl_down_sync(FULL, v.y, 1));
}
__device__ __forceinline__ Belief<float> shfl_up_b(const Belief<float> &b) {
    Belief<float> o;
    o.ehi = __shfl_up_sync(FULL, b.ehi, 1);
    o.elo = __shfl_up_sync(FULL, b.elo, 1);
    o.lhi = __shfl_up_sync(FULL, b.lhi, 1);
    o.llo = __shfl_up_sync(FULL, b.llo, 1);
    return o;
}
__device__ __forceinline__ Belief<float> shfl_down_b(const Belief<float> &b) {
    Belief<float> o;
    o.ehi = __shfl_down_sync(FULL, b.ehi, 1);
    o.elo = __shfl_down_sync(FULL, b.elo, 1);
    o.lhi = __shfl_down_sync(FULL, b.lhi, 1);
    o.llo = __shfl_down_sync(FULL, b.llo, 1);
    return o;
}

// One row as loaded (no shuffles yet, so the loads stay in flight).
struct RowRaw {
    Row5 msg;      // outgoing messages of the row's cell factors at this lane's column
    float2 fx;     // lane 0: E message of column x-1; lane 31: W message of column x+1
    int o0;        // observation index at (x, y)
    int ox;        // lane 0: index at (x-1, y); lane 31: index at (x+1, y)
};

// One row with its x-neighbour terms resolved by shuffles.
struct RowState {
    Row5 msg;
    float2 e_left;   // E message of the factor one column to the left (into this node)
    float2 w_right;  // W message of the factor one column to the right (into this node)
    int o0, o1, om;  // observation index at columns x, x+1 and x-1
};

__device__ __forceinline__ RowRaw load_raw(const DevProblem &p, const float2 *P, int lane, int x, int y) {
    RowRaw r;
    r.msg = load_row(P, p.pn, p.px, p.nx, p.ny, x, y);
    r.fx = make_float2(0.f, 0.f);
    if (lane == 0) r.fx = load_one(P, p.pn, p.px, p.nx, p.ny, DIR_E, x - 1, y);
    if (lane == 31) r.fx = load_one(P, p.pn, p.px, p.nx, p.ny, DIR_W, x + 1, y);
    r.o0 = r.ox = 0;
    if (p.m > 0) {
        r.o0 = load_optr(p.optr, p.nx, p.ny, x, y);
        if (lane == 0) r.ox = load_optr(p.optr, p.nx, p.ny, x - 1, y);
        if (lane == 31) r.ox = load_optr(p.optr, p.nx, p.ny, x + 1, y);
    }
    return r;
}

__device__ __forceinline__ RowState finalize(const RowRaw &r, int lane) {
    RowState s;
    s.msg = r.msg;
    s.e_left = shfl_up2(r.msg.m[DIR_E]);
    s.w_right = shfl_down2(r.msg.m[DIR_W]);
    s.o0 = r.o0;
    s.o1 = __shfl_down_sync(FULL, r.o0, 1);
    s.om = __shfl_up_sync(FULL, r.o0, 1);
    if (lane == 0) {
        s.e_left = r.fx;
        s.om = r.ox;
    }
    if (lane == 31) {
        s.w_right = r.fx;
        s.o1 = r.ox;
    }
    return s;
}

// Compensated belief of node (x, y): `below` is row y-1 (its N messages enter (x, y)), `at` is
// row y, `above_s` is the S message of the factor at (x, y+1).
__device__ __forceinline__ Belief<float> belief_at(const DevProblem &p, const float *O, int x, int y,
                                                  const RowState &below, const RowState &at, float2 above_s) {
    Belief<float> b;
    if (x < 0 || x >= p.nx || y < 0 || y >= p.ny) {
        b.ehi = b.elo = b.lhi = b.llo = 0.f;
        return b;
    }
    float2 m = at.msg.m[DIR_C];
    CompSum<float> se(m.x), sl(m.y);
    if (x > 0) { se.add(at.e_left.x); sl.add(at.e_left.y); }
    if (x < p.nx - 1) { se.add(at.w_right.x); sl.add(at.w_right.y); }
    if (y > 0) { m = below.msg.m[DIR_N]; se.add(m.x); sl.add(m.y); }
    if (y < p.ny - 1) { se.add(above_s.x); sl.add(above_s.y); }
    if (p.m > 0) {
        // bases (x-1, y), (x, y) then (x-1, y-1), (x, y-1): corners 1, 0, 3, 2.  Base cells exist
        // only in columns <= nx-2 and rows <= ny-2 (an index read outside the grid is 0, so the
        // last column's empty range is closed explicitly).
        const bool last = x == p.nx - 1;   // no base cell in the last column: corner-0 range empty
        add_obs_pair(se, sl, O, x > 0 ? at.om : at.o0, at.o0, last ? at.o0 : at.o1, 1, 0);
        if (y > 0) add_obs_pair(se, sl, O, x > 0 ? below.om : below.o0, below.o0, last ? below.o0 : below.o1, 3, 2);
    }
    se.finish();
    sl.finish();
    b.ehi = se.hi; b.elo = se.lo; b.lhi = sl.hi; b.llo = sl.lo;
    return b;
}

constexpr int RING = 16;   // belief rows kept per warp (a power of two >= OBS_BATCH + 1)
constexpr int OBS_BATCH = 8;
constexpr int SWEEP_WARPS = 4;   // warps per block

struct WarpRing {
    Belief<float> bel[RING][32];   // beliefs of the last RING rows, one per lane
    int2 range[RING];              // observations based in the strip's cells of that row
};

// Damped messages of the cell factor (x, r).  `a` holds the row of L for this cell (literal
// -1 entries let the compiler fold the generic update for interior cells; the arithmetic is
// the same either way).
__device__ __forceinline__ void cell_factor(const float (&a)[5], float var_prior, float r, float beta,
                                            const Row5 &own, const Belief<float> *const (&bs)[5],
                                            float2 *Q, int64_t pn, int64_t pc) {
    float lam[5], eta[5];
#pragma unroll
    for (int u = 0; u < 5; ++u) {
        if (a[u] != 0.f) {
            cavity(*bs[u], own.m[u].x, own.m[u].y, eta[u], lam[u]);
        } else {
            lam[u] = 1.f;
            eta[u] = 0.f;
        }
    }
    float L[5], E[5];
    factor_messages<float, 5>(a, var_prior, r, lam, eta, L, E);
#pragma unroll
    for (int u = 0; u < 5; ++u) {
        float2 out;
        if (a[u] != 0.f) {
            out.x = damp(own.m[u].x, E[u], beta);
            out.y = damp(own.m[u].y, L[u], beta);
        } else {
            out.x = 0.f;
            out.y = 0.f;
        }
        __stcs(Q + u * pn + pc, out);
    }
}

// Observation factors based in rows rb..re of the strip, one factor per lane; the beliefs of
// their nodes come from the warp's ring (rows rb..re+1 are there).
__device__ __forceinline__ void obs_batch(const DevProblem &p, const WarpRing &ring, int lane, int x0, int rb,
                                          int re, const float *O, float *OQ, float beta) {
    const int nb = re - rb + 1;   // 1 .. OBS_BATCH rows
    int st = 0, cnt = 0;
    if (lane < nb) {
        const int2 rg = ring.range[(rb + lane) & (RING - 1)];
        st = rg.x;
        cnt = rg.y - rg.x;
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < OBS_BATCH; o <<= 1) {
        const int v = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(FULL, inc, nb - 1);
    const int excl = inc - cnt;
    if (total == 0) return;
    const float *Wt = (const float *)p.ow;
    const float *YV = (const float *)p.ovar;
    for (int j0 = 0; j0 < total; j0 += 32) {
        const int j = j0 + lane;
        int i = 0;
#pragma unroll
        for (int t = 1; t < OBS_BATCH; ++t) {
            const int e = __shfl_sync(FULL, excl, t);
            if (t < nb && e <= j) i = t;
        }
        const int sti = __shfl_sync(FULL, st, i);
        const int exi = __shfl_sync(FULL, excl, i);
        if (j < total) {
            const int row = rb + i;
            const int64_t k = sti + (j - exi);
            const int bx = p.obase[k] - row * p.nx;
            const int lb = bx - x0 + 1;   // lane of the base column
            const Belief<float> *r0 = ring.bel[row & (RING - 1)];
            const Belief<float> *r1 = ring.bel[(row + 1) & (RING - 1)];
            const Belief<float> *ob[4] = {&r0[lb], &r0[lb + 1], &r1[lb], &r1[lb + 1]};
            const float4 w4 = *reinterpret_cast<const float4 *>(Wt + 4 * k);
            const float a4[4] = {w4.x, w4.y, w4.z, w4.w};
            const float4 o01 = *reinterpret_cast<const float4 *>(O + 8 * k);       // (eta, Lambda) x 2
            const float4 o23 = *reinterpret_cast<const float4 *>(O + 8 * k + 4);
            const float oe[4] = {o01.x, o01.z, o23.x, o23.z};
            const float ol[4] = {o01.y, o01.w, o23.y, o23.w};
            float olam[4], oeta[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cavity(*ob[u], oe[u], ol[u], oeta[u], olam[u]);
            float OL[4], OE[4];
            const float2 yv = *reinterpret_cast<const float2 *>(YV + 2 * k);
            factor_messages<float, 4>(a4, yv.y, yv.x, olam, oeta, OL, OE);
            float4 n01, n23;
            n01.x = damp(oe[0], OE[0], beta); n01.y = damp(ol[0], OL[0], beta);
            n01.z = damp(oe[1], OE[1], beta); n01.w = damp(ol[1], OL[1], beta);
            n23.x = damp(oe[2], OE[2], beta); n23.y = damp(ol[2], OL[2], beta);
            n23.z = damp(oe[3], OE[3], beta); n23.w = damp(ol[3], OL[3], beta);
            *reinterpret_cast<float4 *>(OQ + 8 * k) = n01;
            *reinterpret_cast<float4 *>(OQ + 8 * k + 4) = n23;
        }
    }
}

// One strip (30 columns x H rows) of one problem, processed by one warp.
template <int H>
__device__ __forceinline__ void sweep_strip(const DevProblem &p, WarpRing &ring, int lane, int strip, int src,
                                            float beta) {
    const int nx = p.nx, ny = p.ny;
    const int64_t pn = p.pn;
    const int ncs = (nx + SW - 1) / SW;
    const float2 *P = (const float2 *)p.P[src];
    float2 *Q = (float2 *)p.P[src ^ 1];
    const float *O = (const float *)p.O[src];
    float *OQ = (float *)p.O[src ^ 1];
    const float var_prior = p.var_f;
    const float aC_in = p.aC_f[4];

    const int cs = strip % ncs, rs = strip / ncs;
    const int x0 = cs * SW;
    const int x = x0 - 1 + lane;
    const bool owned = lane >= 1 && lane <= SW && x < nx;
    const bool x_inner = x > 0 && x < nx - 1;
    const int y0 = rs * H, y1 = min(y0 + H, ny);
    const int end_lane = min(31, nx - x0);   // lane holding column min(x0 + 30, nx - 1)

    // prologue: beliefs of rows y0-1 and y0; raw rows y0+1 .. y0+3 in flight
    const RowState s_m2 = finalize(load_raw(p, P, lane, x, y0 - 2), lane);
    const RowState s_m1 = finalize(load_raw(p, P, lane, x, y0 - 1), lane);
    RowState s_0 = finalize(load_raw(p, P, lane, x, y0), lane);
    RowRaw r1 = load_raw(p, P, lane, x, y0 + 1);
    RowRaw r2 = load_raw(p, P, lane, x, y0 + 2);
    RowRaw r3 = load_raw(p, P, lane, x, y0 + 3);
    Belief<float> b_prev = belief_at(p, O, x, y0 - 1, s_m2, s_m1, s_0.msg.m[DIR_S]);
    Belief<float> b_cur = belief_at(p, O, x, y0, s_m1, s_0, r1.msg.m[DIR_S]);
    __syncwarp();   // the ring may still be read by the previous strip's last batch
    ring.bel[y0 & (RING - 1)][lane] = b_cur;

    for (int r = y0; r < y1; ++r) {
        const RowRaw r4 = load_raw(p, P, lane, x, r + 4);   // in flight for three rows
        const RowState s_1 = finalize(r1, lane);
        const Belief<float> b_next = belief_at(p, O, x, r + 1, s_0, s_1, r2.msg.m[DIR_S]);
        ring.bel[(r + 1) & (RING - 1)][lane] = b_next;
        if (p.m > 0) {
            const int st = __shfl_sync(FULL, s_0.o0, 1);
            const int en = __shfl_sync(FULL, s_0.o0, end_lane);
            if (lane == 0) ring.range[r & (RING - 1)] = make_int2(st, en > st ? en : st);
        }

        const Belief<float> b_w = shfl_up_b(b_cur);
        const Belief<float> b_e = shfl_down_b(b_cur);
        if (owned) {
            const Belief<float> *const bs[5] = {&b_cur, &b_w, &b_e, &b_prev, &b_next};
            const int64_t c = (int64_t)r * nx + x, pc = (int64_t)r * p.px + x;
            const float tg = p.ptgt ? ((const float *)p.ptgt)[c] : 0.f;
            if (x_inner && r > 0 && r < ny - 1) {
                const float a[5] = {aC_in, -1.f, -1.f, -1.f, -1.f};
                cell_factor(a, var_prior, tg, beta, s_0.msg, bs, Q, pn, pc);
            } else {
                const int deg = grid_degree(r, x, nx, ny);
                const float a[5] = {p.aC_f[deg], x > 0 ? -1.f : 0.f, x < nx - 1 ? -1.f : 0.f,
                                    r > 0 ? -1.f : 0.f, r < ny - 1 ? -1.f : 0.f};
                cell_factor(a, var_prior, tg, beta, s_0.msg, bs, Q, pn, pc);
            }
        }
        if (p.m > 0 && ((r - y0) % OBS_BATCH == OBS_BATCH - 1 || r == y1 - 1)) {
            __syncwarp();
            const int rb = r - (r - y0) % OBS_BATCH;
            obs_batch(p, ring, lane, x0, rb, r, O, OQ, beta);
            __syncwarp();
        }
        b_prev = b_cur;
        b_cur = b_next;
        s_0 = s_1;
        r1 = r2;
        r2 = r3;
        r3 = r4;
    }
}

template <int H>
__global__ void __launch_bounds__(SWEEP_WARPS * 32) k_sweep(DevProblem p, int src, float beta) {
    __shared__ WarpRing rings[SWEEP_WARPS];
    const int lane = threadIdx.x & 31;
    WarpRing &ring = rings[threadIdx.x >> 5];
    const int nstrips = ((p.nx + SW - 1) / SW) * ((p.ny + H - 1) / H);
    for (int strip = blockIdx.x * SWEEP_WARPS + (threadIdx.x >> 5); strip < nstrips;
         strip += gridDim.x * SWEEP_WARPS)
        sweep_strip<H>(p, ring, lane, strip, src, beta);
}

// Many independent problems in one persistent launch: the strips of all problems form one work
// list (strip_start[i] = first strip of problem i, prefix over the problems), taken by the warps
// of a grid sized to fill the GPU.  Problems whose active flag is 0 are skipped (their messages
// stay as they are).  All problems share the ping-pong parity `src`.
template <int H>
__global__ void __launch_bounds__(SWEEP_WARPS * 32)
    k_sweep_batch(const DevProblem *__restrict__ table, const int *__restrict__ strip_start,
                  const int *__restrict__ active, int count, int src, float beta) {
    __shared__ WarpRing rings[SWEEP_WARPS];
    const int lane = threadIdx.x & 31;
    WarpRing &ring = rings[threadIdx.x >> 5];
    const int total = strip_start[count];
    for (int g = blockIdx.x * SWEEP_WARPS + (threadIdx.x >> 5); g < total; g += gridDim.x * SWEEP_WARPS) {
        int lo = 0, hi = count - 1;   // last problem whose first strip is <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (strip_start[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        if (!active[lo]) continue;
        sweep_strip<H>(table[lo], ring, lane, g - strip_start[lo], src, beta);
    }
}

template <int H> cudaError_t launch_h(const DevProblem &p, int src, double beta, cudaStream_t st) {
    static int grid_cache = 0, configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        int nsm = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<H>, SWEEP_WARPS * 32, 0);
        if (e != cudaSuccess) return e;
        grid_cache = nsm * (per_sm > 0 ? per_sm : 1);
        configured_dev = dev;
    }
    const int nstrips = ((p.nx + SW - 1) / SW) * ((p.ny + H - 1) / H);
    const int blocks = (nstrips + SWEEP_WARPS - 1) / SWEEP_WARPS;
    const int grid = blocks < grid_cache ? blocks : grid_cache;
    k_sweep<H><<<grid, SWEEP_WARPS * 32, 0, st>>>(p, src, (float)beta);
    return cudaGetLastError();
}

}  // namespace

bool sweep_shape_supported(int h) { return h == 16 || h == 32 || h == 64 || h == 128; }

int sweep_strips(int nx, int ny, int h) { return ((nx + SW - 1) / SW) * ((ny + h - 1) / h); }

namespace {
template <int H>
cudaError_t launch_batch_h(const DevProblem *table, const int *strip_start, const int *active, int count,
                           int total_strips, int src, double beta, cudaStream_t st) {
    static int grid_cache = 0, configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        int nsm = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_batch<H>, SWEEP_WARPS * 32, 0);
        if (e != cudaSuccess) return e;
        grid_cache = nsm * (per_sm > 0 ? per_sm : 1);
        configured_dev = dev;
    }
    const int blocks = (total_strips + SWEEP_WARPS - 1) / SWEEP_WARPS;
    const int grid = blocks < grid_cache ? blocks : grid_cache;
    if (grid < 1) return cudaSuccess;
    k_sweep_batch<H><<<grid, SWEEP_WARPS * 32, 0, st>>>(table, strip_start, active, count, src, (float)beta);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_sweep_batch(const DevProblem *table, const int *strip_start, const int *active, int count,
                               int total_strips, int src, double beta, int h, cudaStream_t st) {
    switch (h) {
        case 16: return launch_batch_h<16>(table, strip_start, active, count, total_strips, src, beta, st);
        case 32: return launch_batch_h<32>(table, strip_start, active, count, total_strips, src, beta, st);
        case 64: return launch_batch_h<64>(table, strip_start, active, count, total_strips, src, beta, st);
        case 128: return launch_batch_h<128>(table, strip_start, active, count, total_strips, src, beta, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_iteration(const DevProblem &p, int src, double beta, int h, cudaStream_t st) {
    if (p.prec != 0) return cudaErrorInvalidValue;
    switch (h) {
        case 16: return launch_h<16>(p, src, beta, st);
        case 32: return launch_h<32>(p, src, beta, st);
        case 64: return launch_h<64>(p, src, beta, st);
        case 128: return launch_h<128>(p, src, beta, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gabp
