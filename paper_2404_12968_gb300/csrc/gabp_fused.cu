// Fused GaBP iteration: one kernel computes the beliefs and every factor update of one
// synchronous iteration (Alg. 2, "Iterate MP Until Convergence": all new messages from the
// previous iteration's messages), so each message is read from HBM once and written once.
//
// Work unit: a TX x TY tile of cells.  The block
//   1. stages the 5 prior-message planes over the tile plus a 2-cell halo in shared memory
//      (the halo reads of neighbouring tiles hit L2, not HBM);
//   2. computes the compensated beliefs of the tile plus a 1-cell halo (every node a factor of
//      the tile touches), adding the observation messages that target those nodes;
//   3. updates the tile's cell factors (prior) and the observation factors whose base cell lies
//      in the tile, and writes the damped messages to the other ping-pong buffer.
// The arithmetic and the summation order are those of the split kernels, so both paths give
// bit-identical messages.
#include "gabp_device.cuh"
#include "gabp_internal.h"

namespace gabp {

namespace {

constexpr int FT = 256;   // threads per block

template <typename T, int TX, int TY> struct FusedLayout {
    static constexpr int RX = TX + 4, RY = TY + 4;   // staged message window (2-cell halo)
    static constexpr int BX = TX + 2, BY = TY + 2;   // belief window (1-cell halo)
    static constexpr size_t msg_bytes = sizeof(T2<T>) * 5 * RX * RY;
    static constexpr size_t bel_bytes = sizeof(Belief<T>) * BX * BY;
    static constexpr size_t bytes = msg_bytes + bel_bytes + sizeof(int) * 2 * (TY + 1);
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(FT) k_fused(DevProblem p, int src, T beta) {
    using LY = FusedLayout<T, TX, TY>;
    constexpr int RX = LY::RX, RY = LY::RY, BX = LY::BX, BY = LY::BY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2<T> *sm = reinterpret_cast<T2<T> *>(smem_raw);                         // [5][RY][RX]
    Belief<T> *sb = reinterpret_cast<Belief<T> *>(smem_raw + LY::msg_bytes); // [BY][BX]
    int *rstart = reinterpret_cast<int *>(smem_raw + LY::msg_bytes + LY::bel_bytes);  // [TY+1]
    int *rpre = rstart + (TY + 1);                                                     // [TY+1]

    const int nx = p.nx, ny = p.ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const T2<T> *P = (const T2<T> *)p.P[src];
    T2<T> *Q = (T2<T> *)p.P[src ^ 1];
    const T *O = (const T *)p.O[src];
    T *OQ = (T *)p.O[src ^ 1];
    const int *optr = p.optr;

    // 1. stage the message window
    for (int q = threadIdx.x; q < 5 * RX * RY; q += FT) {
        const int d = q / (RX * RY);
        const int rem = q - d * (RX * RY);
        const int ly = rem / RX, lx = rem - ly * RX;
        const int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        T2<T> val;
        val.x = T(0);
        val.y = T(0);
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) val = P[d * p.pn + (int64_t)gy * p.px + gx];
        sm[q] = val;
    }
    // observation ranges of the tile's base rows (cells [x0, x0+TX) of rows y0 .. y0+TY-1)
    if (p.m > 0 && threadIdx.x <= TY) {
        const int r = threadIdx.x;
        const int gy = y0 + r;
        int lo = 0, cnt = 0;
        if (r < TY && gy < ny) {
            const int xe = min(x0 + TX, nx);
            lo = optr[(int64_t)gy * nx + x0];
            cnt = optr[(int64_t)gy * nx + xe] - lo;
        }
        rstart[r] = lo;
        rpre[r] = cnt;   // prefix taken below
    }
    __syncthreads();
    if (p.m > 0 && threadIdx.x == 0) {
        int acc = 0;
        for (int r = 0; r < TY; ++r) {
            const int c = rpre[r];
            rpre[r] = acc;
            acc += c;
        }
        rpre[TY] = acc;
    }

    // 2. compensated beliefs over the tile plus a 1-cell halo
    for (int q = threadIdx.x; q < BX * BY; q += FT) {
        const int ly = q / BX, lx = q - ly * BX;
        const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
        const int rx = lx + 1, ry = ly + 1;
        const int64_t v = (int64_t)gy * nx + gx;
        T2<T> m = sm[(DIR_C * RY + ry) * RX + rx];
        CompSum<T> se(m.x), sl(m.y);
        if (gx > 0) { m = sm[(DIR_E * RY + ry) * RX + rx - 1]; se.add(m.x); sl.add(m.y); }
        if (gx < nx - 1) { m = sm[(DIR_W * RY + ry) * RX + rx + 1]; se.add(m.x); sl.add(m.y); }
        if (gy > 0) { m = sm[(DIR_N * RY + ry - 1) * RX + rx]; se.add(m.x); sl.add(m.y); }
        if (gy < ny - 1) { m = sm[(DIR_S * RY + ry + 1) * RX + rx]; se.add(m.x); sl.add(m.y); }
        if (p.m > 0) {
            add_obs_pair(se, sl, O, gx > 0 ? optr[v - 1] : optr[v], optr[v], optr[v + 1], 1, 0);
            if (gy > 0)
                add_obs_pair(se, sl, O, gx > 0 ? optr[v - nx - 1] : optr[v - nx], optr[v - nx], optr[v - nx + 1], 3, 2);
        }
        se.finish();
        sl.finish();
        Belief<T> b;
        b.ehi = se.hi; b.elo = se.lo; b.lhi = sl.hi; b.llo = sl.lo;
        sb[q] = b;
    }
    __syncthreads();

    // 3a. prior cell factors of the tile
    const T var_prior = prior_var<T>(p);
    for (int q = threadIdx.x; q < TX * TY; q += FT) {
        const int ty = q / TX, tx = q - ty * TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= nx || gy >= ny) continue;
        const int64_t c = (int64_t)gy * nx + gx;
        const int deg = grid_degree(gy, gx, nx, ny);
        const T a[5] = {cell_coef<T>(p, deg), gx > 0 ? T(-1) : T(0), gx < nx - 1 ? T(-1) : T(0),
                        gy > 0 ? T(-1) : T(0), gy < ny - 1 ? T(-1) : T(0)};
        // belief-window coordinates of the 5 nodes (C, W, E, S, N)
        const int bxs[5] = {tx + 1, tx, tx + 2, tx + 1, tx + 1};
        const int bys[5] = {ty + 1, ty + 1, ty + 1, ty, ty + 2};
        T2<T> own[5];
        T lam[5], eta[5];
#pragma unroll
        for (int u = 0; u < 5; ++u) {
            own[u] = sm[(u * RY + ty + 2) * RX + tx + 2];
            if (a[u] != T(0)) {
                cavity(sb[bys[u] * BX + bxs[u]], own[u].x, own[u].y, eta[u], lam[u]);
            } else {
                lam[u] = T(1);
                eta[u] = T(0);
            }
        }
        T L[5], E[5];
        const T r = p.ptgt ? ((const T *)p.ptgt)[c] : T(0);
        factor_messages<T, 5>(a, var_prior, r, lam, eta, L, E);
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
            Q[u * p.pn + (int64_t)gy * p.px + gx] = out;
        }
    }

    // 3b. observation factors whose base cell lies in the tile
    if (p.m > 0) {
        const int total = rpre[TY];
        const T *W = (const T *)p.ow;
        const T *YV = (const T *)p.ovar;
        for (int q = threadIdx.x; q < total; q += FT) {
            int r = 0;
            while (r + 1 < TY && rpre[r + 1] <= q) ++r;
            const int64_t k = rstart[r] + (q - rpre[r]);
            const int b = p.obase[k];
            const int by = b / nx, bx = b - by * nx;
            const int lx = bx - x0 + 1, ly = by - y0 + 1;   // belief-window coordinates
            const int bidx[4] = {ly * BX + lx, ly * BX + lx + 1, (ly + 1) * BX + lx, (ly + 1) * BX + lx + 1};
            const T a[4] = {W[4 * k], W[4 * k + 1], W[4 * k + 2], W[4 * k + 3]};
            T oe[4], ol[4], lam[4], eta[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                oe[u] = O[8 * k + 2 * u];
                ol[u] = O[8 * k + 2 * u + 1];
                cavity(sb[bidx[u]], oe[u], ol[u], eta[u], lam[u]);
            }
            T L[4], E[4];
            factor_messages<T, 4>(a, YV[2 * k + 1], YV[2 * k], lam, eta, L, E);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                OQ[8 * k + 2 * u] = damp(oe[u], E[u], beta);
                OQ[8 * k + 2 * u + 1] = damp(ol[u], L[u], beta);
            }
        }
    }
}

template <typename T, int TX, int TY>
cudaError_t launch_shape(const DevProblem &p, int src, double beta, cudaStream_t st) {
    using LY = FusedLayout<T, TX, TY>;
    static bool configured = false;   // per instantiation; the attribute is per function
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<T, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((unsigned)((p.nx + TX - 1) / TX), (unsigned)((p.ny + TY - 1) / TY));
    k_fused<T, TX, TY><<<grid, FT, LY::bytes, st>>>(p, src, (T)beta);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const DevProblem &p, int src, double beta, FusedShape s, cudaStream_t st) {
#define GABP_SHAPE(X, Y) \
    if (s.tx == X && s.ty == Y) return launch_shape<T, X, Y>(p, src, beta, st);
    GABP_SHAPE(32, 8)
    GABP_SHAPE(32, 16)
    GABP_SHAPE(64, 8)
    GABP_SHAPE(64, 16)
    GABP_SHAPE(128, 8)
    GABP_SHAPE(32, 32)
#undef GABP_SHAPE
    return cudaErrorInvalidValue;
}

}  // namespace

bool fused_shape_supported(int tx, int ty) {
    return (tx == 32 && (ty == 8 || ty == 16 || ty == 32)) || (tx == 64 && (ty == 8 || ty == 16)) ||
           (tx == 128 && ty == 8);
}

size_t fused_smem_bytes(int prec, FusedShape s) {
    const size_t t2 = prec ? 16 : 8, bel = prec ? 32 : 16;
    return t2 * 5 * (s.tx + 4) * (s.ty + 4) + bel * (s.tx + 2) * (s.ty + 2) + sizeof(int) * 2 * (s.ty + 1);
}

cudaError_t launch_fused_iteration(const DevProblem &p, int src, double beta, FusedShape shape,
                                   cudaStream_t st) {
    return p.prec ? dispatch<double>(p, src, beta, shape, st) : dispatch<float>(p, src, beta, shape, st);
}

}  // namespace gabp
