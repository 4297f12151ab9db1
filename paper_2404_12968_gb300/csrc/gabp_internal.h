// Internal interface between the host engine (gabp_api.cu) and the kernel translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace gabp {

// Device-resident description of one problem instance.  All pointers are device pointers.
// Message buffers are typed by the precision (float or double) of the instance.
struct DevProblem {
    int nx, ny;
    int64_t n, m;
    int prec;            // 0 = FP32, 1 = FP64
    double gamma;        // prior scale (factor precision of every cell factor)
    double aC[5];        // kappa^2 + deg for deg = 0..4 (FP64)
    float var_f;         // (float)(1 / gamma), rounded once on the host
    float aC_f[5];       // (float)aC[d]
    float aC_lo[5];      // aC[d] - aC_f[d] rounded: aC[d] as a double-float pair (aC_f, aC_lo)
    float gam_hi, gam_lo;   // gamma as a double-float pair
    float l2c_f[5];      // alpha = 4: centre coefficient (kappa^2 + d)^2 + d of a cell of degree d, as float
    float l2n_f[25];     // alpha = 4: neighbour coefficient -(aC[dc] + aC[du]) for degrees (dc, du), as float
    float init_c_f[5];   // cold-start precision gamma aC[d]^2 of a centre slot of degree d, as float
    float init_n_f;      // cold-start precision gamma (-1)^2 of a neighbour slot, as float
    const float2 *owdf;  // FP32 contexts: 4 * m observation weights as double-float (hi, lo) pairs
    const float2 *oysdf; // FP32 contexts: 2 * m (y, 1/sigma^2) as double-float pairs
    void *P[2];          // prior messages, ping-pong: planes * pn (eta, Lambda) pairs
    // layout of the prior message planes: node (i, j) of plane d at d * pn + i * px + j.  px = nx
    // except for the members of a batch with an odd width, whose rows are padded to px = nx + 1
    // so that every row starts on a 16-byte boundary (tensor copies); the padding cells hold
    // (0, 0) in both buffers.  pn = px * ny.
    int px;
    int64_t pn;
    void *O[2];          // observation messages, ping-pong: per observation (eta, Lambda) of corners 0..3, interleaved
    const int *obase;    // m base-cell indices (sorted ascending)
    const void *ow;      // 4 * m bilinear weights (T)
    const void *ovar;    // 2 * m (y, sigma^2) pairs (T)
    const double *ow64;  // 4 * m weights, FP64 (residual)
    const double *oys64; // 2 * m (y, 1/sigma^2) pairs, FP64 (residual)
    const int *optr;     // n + 1: observations with base cell c are optr[c] .. optr[c+1]-1
    void *belief;        // n compensated beliefs (4 T each), split kernels only
    double *mu64;        // n, residual scratch
    double *z64;         // n, residual scratch
    double *e64;         // m, residual scratch
    double *part;        // residual partial sums (RES_BLOCKS)
    double *scal;        // 2 doubles: [0] = ||r||^2, [1] = ||b||^2
    int *err;            // device error flag (a bounded wait in a kernel gave up)
    int debug_stall;     // test hook: the TMA kernel first waits on a barrier nothing completes
    int order;           // prior operator: 1 = L (alpha = 2, 5-slot cell factors), 2 = L^2 (alpha = 4)
    int planes;          // prior message planes: 5 (order 1) or 13 (order 2)
    // targets r_c of the cell factors exp(-(gamma / 2) (l_c . f - r_c)^2), r = L f_b for a prior
    // mean f_b (NULL: every target is zero, the zero prior mean): in the message precision for
    // the iteration kernels, in FP64 for the residual and ||b||, and as double-float pairs for
    // the residual of FP32 contexts
    const void *ptgt;
    const double *ptgt64;
    const float2 *ptgtdf;
};

// plane index of node (i, j)
__host__ __device__ __forceinline__ int64_t plane_at(const DevProblem &p, int i, int j) {
    return (int64_t)i * p.px + j;
}

// Prior constants in the kernel's precision.  FP32 kernels read the values rounded once on the
// host (the same roundings as converting the FP64 values on the device, without FP64
// instructions in the FP32 kernels); FP64 kernels read the FP64 values.
template <typename T> __device__ __forceinline__ T prior_var(const DevProblem &p);
template <> __device__ __forceinline__ float prior_var<float>(const DevProblem &p) { return p.var_f; }
template <> __device__ __forceinline__ double prior_var<double>(const DevProblem &p) { return 1.0 / p.gamma; }
template <typename T> __device__ __forceinline__ T cell_coef(const DevProblem &p, int deg);
template <> __device__ __forceinline__ float cell_coef<float>(const DevProblem &p, int deg) { return p.aC_f[deg]; }
template <> __device__ __forceinline__ double cell_coef<double>(const DevProblem &p, int deg) { return p.aC[deg]; }

constexpr int RES_BLOCKS = 1024;   // fixed partition of the deterministic residual reduction

// ---- split path (gabp_split.cu) ----
cudaError_t launch_split_iteration(const DevProblem &p, int src, double beta, cudaStream_t st);
cudaError_t launch_beliefs(const DevProblem &p, int src, cudaStream_t st);
cudaError_t launch_init_cold(const DevProblem &p, int dst, int paper, cudaStream_t st);
cudaError_t launch_init_warm(const DevProblem &p, int dst, const double *mu0, const double *lam0,
                             cudaStream_t st);
cudaError_t launch_obs_precompute(const DevProblem &p, const double *raw_xy, const double *raw_y,
                                  const double *raw_var, cudaStream_t st);
cudaError_t launch_rhs_norm(const DevProblem &p, cudaStream_t st);   // scal[1] = ||b||^2
// optr[c] = number of observations with base cell < c (c = 0 .. n), from the sorted obase
cudaError_t launch_obs_pointers(const DevProblem &p, cudaStream_t st);
// ---- observation layout (gabp_obs_sort.cu) ----
// Base cells of m observations at xy (device, input order; validated: inside the grid) and their
// stable sort by base cell: obase (m ints) = the sorted base cells; sxy (2 m), sy, svar (m each)
// = the raw data in that order.  scratch: obs_sort_scratch_bytes(m) bytes of device memory.
size_t obs_sort_scratch_bytes(int64_t m);
cudaError_t launch_obs_sort(int64_t m, int nx, int ny, const double *xy, const double *y, const double *var,
                            int *obase, double *sxy, double *sy, double *svar, void *scratch, cudaStream_t st);
// residual of the messages in buffer src; leaves ||r||^2 in scal[0] (beliefs recomputed)
cudaError_t launch_residual(const DevProblem &p, int src, cudaStream_t st);
// ---- the alpha = 4 prior (order 2: cell factors = rows of L^2, 13 planes; gabp_split.cu) ----
// one synchronous iteration (beliefs, cell factors, observation factors); initialisation as
// launch_init_cold (which dispatches on p.order, as do launch_beliefs, launch_residual and
// launch_msg_change)
cudaError_t launch_l2_iteration(const DevProblem &p, int src, double beta, cudaStream_t st);
// the same iteration as one fused FP32 kernel (gabp_fused_l2.cu): 28 x ty tiles (ty = 4 or 8),
// runs of `run` tiles down a tile column; messages bit-identical to the split kernels'.
// fused_l2_choose_run: the run length (1..16) that balances the persistent blocks for p.
bool fused_l2_shape_supported(int ty);
int fused_l2_choose_run(const DevProblem &p, int ty);
cudaError_t launch_fused_l2_iteration(const DevProblem &p, int ty, int run, int src, double beta, cudaStream_t st);
// ---- the paper's pairwise re-weighted form (gabp_pairwise.cu) ----
// coefficients P_ii (n), h (n), P_{i, i + off_d} (12 n) in the context's precision; messages are
// 12 n (a, b) pairs per buffer
cudaError_t pw_setup(const DevProblem &p, void *Pd, void *hv, void *Pn, cudaStream_t st);
cudaError_t pw_zero(const DevProblem &p, void *msg, cudaStream_t st);
// Alg. 2 around the pairwise form: directed edges (pairs within the 12 offsets); the mean
// |m_a - m_b| numerator over both message buffers (nparts partial sums in part, total in *out);
// "Upscale Messages" from a coarse level's messages to the next finer level's
int64_t pw_edge_count(int nx, int ny);
cudaError_t pw_change(const DevProblem &p, const void *a, const void *b, double *part, int nparts, double *out,
                      cudaStream_t st);
cudaError_t pw_upscale(const DevProblem &fine, const DevProblem &coarse, const void *coarse_msg, void *fine_msg,
                       cudaStream_t st);
cudaError_t pw_iterate(const DevProblem &p, const void *Pd, const void *hv, const void *Pn, const void *src, void *dst,
                       double c, double eta, cudaStream_t st);
// marginals into mean / var (FP64, var may be NULL), or (to_residual) the mean into p.mu64
cudaError_t pw_marginals(const DevProblem &p, const void *Pd, const void *hv, const void *msg, double c, double *mean,
                         double *var, int to_residual, cudaStream_t st);
// residual of the mean already in p.mu64 (double-float pairs for FP32 contexts, FP64 otherwise)
cudaError_t launch_residual_mu(const DevProblem &p, cudaStream_t st);
// marginal means (and variances) into mean / var (device addresses; pinned host memory through
// its device address).  direct: each node's belief formed in registers and the outputs written
// at once (for outputs in device memory); otherwise the beliefs are stored first, so that a
// kernel writing across the host link does not also hold the belief sums
cudaError_t launch_marginals(const DevProblem &p, int src, double *mean, double *var,
                             cudaStream_t st, bool direct = true);

// ---- learned warm start (gabp_split.cu kernels, network in gabp_wsnet.cu) ----
cudaError_t launch_ws_input(const DevProblem &p, double scale, double kappa, int Hp, int Wp, void *x, cudaStream_t st);
cudaError_t launch_ws_target(const DevProblem &p, int src, double scale, int Hp, int Wp, float *t, cudaStream_t st);
// multigrid: marginals of the finer grid copied from parent nodes (i >> shift, j >> shift); q_c
// variances or precisions, the output precisions
cudaError_t launch_upscale(const double *mu_c, const double *q_c, int q_is_var, int shift, int nxc, int nyc, int nxf,
                           int nyf, double *mu_f, double *lam_f, cudaStream_t st);
// FP32 contexts: warm-start messages from marginals in FP32 arithmetic; nm: n float2 scratch
cudaError_t launch_init_warm_f32(const DevProblem &p, int dst, const double *mu0, const double *lam0, float2 *nm,
                                 cudaStream_t st);
// FP32 contexts: decode the network output and initialise the messages (dst buffer) in FP32;
// nm: n float2 scratch
cudaError_t launch_ws_init_f32(const DevProblem &p, int dst, double scale, int Wp, const float *out, float2 *nm,
                               cudaStream_t st);
// sum over every stored message component of |m_t - m_{t-1}| (buffers cur and cur ^ 1) into *out
cudaError_t launch_msg_change(const DevProblem &p, int cur, double *out, cudaStream_t st);
// FP32 contexts: double-float (hi, lo) copies of the FP64 observation weights and (y, 1/sigma^2)
cudaError_t launch_df_precompute(const DevProblem &p, cudaStream_t st);
cudaError_t launch_ws_decode(const DevProblem &p, double scale, int Wp, const float *out, double *mu0, double *lam0,
                             cudaStream_t st);
// ---- prior mean (gabp_split.cu) ----
// cell-factor targets t = L d (d: n doubles; NULL = zero) into t64 (FP64), tT (message
// precision) and, for FP32 contexts, tdf (double-float pairs)
cudaError_t launch_cell_targets(const DevProblem &p, const double *d, double *t64, void *tT, float2 *tdf,
                                cudaStream_t st);


// ---- fused path (gabp_fused.cu) ----
struct FusedShape {
    int tx, ty;   // tile in cells
};
bool fused_shape_supported(int tx, int ty);
cudaError_t launch_fused_iteration(const DevProblem &p, int src, double beta, FusedShape shape,
                                   cudaStream_t st);
size_t fused_smem_bytes(int prec, FusedShape shape);

// ---- warp-synchronous column sweep, FP32 (gabp_sweep.cu); tile 30 columns x h rows ----
bool sweep_shape_supported(int h);
cudaError_t launch_sweep_iteration(const DevProblem &p, int src, double beta, int h, cudaStream_t st);
int sweep_strips(int nx, int ny, int h);
// all problems of a batch in one persistent launch (FP32 problems; table/strip_start/active on device)
cudaError_t launch_sweep_batch(const DevProblem *table, const int *strip_start, const int *active, int count,
                               int total_strips, int src, double beta, int h, cudaStream_t st);

// ---- TMA-fed persistent fused path, FP32 (gabp_fused_tma.cu) ----
struct TmaMaps {
    CUtensorMap planes[2];   // message planes of buffer 0 / 1
    CUtensorMap optr;        // observations-by-base-cell index
    int tx = 0, ty = 0;
    int run = 1;             // tiles per run of the single-problem schedule (1..8)
    bool valid = false;
};
// Batched TMA iteration: the work items are the tiles of the active problems, item k (k <
// *nitems) being tile column items[k].y, tile row items[k].z of problem items[k].x; items[k].w
// = 1 when item k - G (the same block's previous item, G blocks) is the tile directly above it
// in the same problem, so that two belief rows carry over.  Every problem's tensor maps sit in
// a global array (CUtensorMap's own alignment; zero for a problem whose rows are not 16-byte
// strided).  *err is raised if a bounded wait ran out.
struct TmaMapsGlobal {
    CUtensorMap planes[2];
    CUtensorMap optr;
};
struct TmaBatchArgs {
    const TmaMapsGlobal *maps;
    const DevProblem *table;
    const int4 *items;
    const int *nitems;
    int *err;
    int debug_stall;   // test hook, as DevProblem::debug_stall
};
bool tma_batch_shape_supported(int ty);   // tile heights of the batched TMA kernel (14, 22, 30)
int tma_batch_grid(int ty, int max_tiles);  // blocks of its launch (0 on error)
cudaError_t launch_tma_batch(const TmaBatchArgs &ba, const DevProblem &first, int ty, int max_tiles, int src,
                             double beta, cudaStream_t st);
bool tma_shape_supported(int tx, int ty);
bool tma_problem_supported(const DevProblem &p);
// parts: which maps to encode (planes need nx even, the observation index nx a multiple of 4)
constexpr int TMA_MAP_PLANES = 1, TMA_MAP_OPTR = 2;
// optr / optr_pitch: a copy of the observation index with rows optr_pitch ints apart (a multiple
// of 4) to encode instead of p.optr (whose rows are nx ints apart).
cudaError_t make_tma_maps(const DevProblem &p, int tx, int ty, TmaMaps &maps, int parts = TMA_MAP_PLANES | TMA_MAP_OPTR,
                          const int *optr = nullptr, int optr_pitch = 0);
size_t tma_smem_bytes(int tx, int ty);
// Tiles per run for a problem on 30 x ty tiles: the length in 1..4 that balances the
// persistent blocks best (longest on ties).
int tma_choose_run(const DevProblem &p, int ty);
cudaError_t launch_tma_iteration(const DevProblem &p, const TmaMaps &maps, int src, double beta,
                                 cudaStream_t st);

}  // namespace gabp

struct gabp_wsnet;
namespace gabp {
int wsnet_forward_device(gabp_wsnet *net, const void *x, int B, int H, int W, float **out, cudaStream_t st,
                         std::string &err);
int wsnet_device(const gabp_wsnet *net);
int wsnet_take_device_error(gabp_wsnet *net);
}  // namespace gabp
