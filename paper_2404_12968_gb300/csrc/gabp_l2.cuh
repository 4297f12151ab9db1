// The alpha = 4 prior's cell factors (Sec. 3.1 with alpha / 2 = 2; App. C, powers of the
// operator): slot offsets and coefficients, shared by the split kernels (gabp_split.cu) and the
// fused FP32 tile kernel (gabp_fused_l2.cu).
#pragma once
#include "gabp_device.cuh"
#include "gabp_internal.h"

namespace gabp {

// The operator matrix is L^2 and cell c's factor has a = row c of L^2 over 13 slots: the cell,
// its 4 neighbours, the 4 diagonal neighbours and the 4 nodes two steps away.  Plane d holds
// the message of cell c's factor to node c + offset(d).  Row c of L^2 = sum_w L_cw L_w.:
// centre (kappa^2 + deg c)^2 + deg c; neighbour u: -(kappa^2 + deg c) - (kappa^2 + deg u)
// (the two one-step paths through c and u); diagonal: 2 (two paths); two steps away: 1.
constexpr int L2_SLOTS = 13;
__host__ __device__ constexpr int l2_dx(int d) {
    return d == 1 || d == 5 || d == 7 ? -1 : d == 2 || d == 6 || d == 8 ? 1 : d == 9 ? -2 : d == 10 ? 2 : 0;
}
__host__ __device__ constexpr int l2_dy(int d) {
    return d == 3 || d == 5 || d == 6 ? -1 : d == 4 || d == 7 || d == 8 ? 1 : d == 11 ? -2 : d == 12 ? 2 : 0;
}

// slot d of cell (i, j)'s factor has its node inside the grid
__device__ __forceinline__ bool l2_in(const DevProblem &p, int i, int j, int d) {
    const int y = i + l2_dy(d), x = j + l2_dx(d);
    return x >= 0 && x < p.nx && y >= 0 && y < p.ny;
}

// coefficient of slot d of cell (i, j)'s factor; 0 if the slot's node is outside the grid
__device__ __forceinline__ double l2_coef(const DevProblem &p, int i, int j, int d) {
    const int nx = p.nx, ny = p.ny;
    const int y = i + l2_dy(d), x = j + l2_dx(d);
    if (x < 0 || x >= nx || y < 0 || y >= ny) return 0.0;
    if (d == 0) {
        const int dc = grid_degree(i, j, nx, ny);
        return p.aC[dc] * p.aC[dc] + (double)dc;
    }
    if (d <= 4) return -(p.aC[grid_degree(i, j, nx, ny)] + p.aC[grid_degree(y, x, nx, ny)]);
    return d <= 8 ? 2.0 : 1.0;
}

// The same coefficient in the kernel's precision.  FP32: from the float tables rounded once on
// the host (the value of l2_coef rounded to float), so the FP32 kernels hold no FP64
// instruction; INTERIOR: every slot's node exists and every degree is 4.
template <typename T, bool INTERIOR>
__device__ __forceinline__ T l2_coef_t(const DevProblem &p, int i, int j, int d) {
    if constexpr (sizeof(T) == 8) {
        return l2_coef(p, i, j, d);
    } else {
        if (d >= 9) return INTERIOR ? 1.f : (l2_in(p, i, j, d) ? 1.f : 0.f);
        if (d >= 5) return INTERIOR ? 2.f : (l2_in(p, i, j, d) ? 2.f : 0.f);
        if (INTERIOR) return d == 0 ? p.l2c_f[4] : p.l2n_f[24];
        if (!l2_in(p, i, j, d)) return 0.f;
        const int dc = grid_degree(i, j, p.nx, p.ny);
        if (d == 0) return p.l2c_f[dc];
        return p.l2n_f[5 * dc + grid_degree(i + l2_dy(d), j + l2_dx(d), p.nx, p.ny)];
    }
}

}  // namespace gabp
