// Host engine and C ABI of libgabp (declared in include/gabp.h).
//
// A context owns the device buffers of one problem: ping-pong message buffers, the sorted
// observation data, the residual scratch.  Iterations run as CUDA-graph replays of a chunk
// of fused (or split) iteration kernels on the context's stream.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "gabp.h"
#include "gabp_internal.h"
#include <nvtx3/nvToolsExt.h>

namespace {
// NVTX range around a public call (header-only NVTX 3: a no-op unless a profiler is attached),
// so that a timeline shows create / iterate / residual / marginals / warm-start phases
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

using gabp::DevProblem;

struct gabp_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap = nullptr;   // private stream used only for graph capture
    DevProblem p{};
    gabp_options opt{};
    int kernel = GABP_KERNEL_FUSED;
    gabp::FusedShape shape{64, 16};
    gabp::TmaMaps maps;
    int l2_run = 0;               // alpha = 4 fused kernel: tiles per run
    int cur = 0;                  // buffer holding the current messages
    int64_t iters = 0;
    double last_res = NAN;
    int64_t edges = 0;
    double bytes_per_iter = 0.0;
    std::string err;
    std::vector<std::pair<void *, bool>> allocs;   // device buffers (pointer, from the pool)
    double *stage = nullptr;      // 2 n doubles of device staging for host <-> device transfers
    double *hscal = nullptr;      // pinned host copy of p.scal
    cudaGraphExec_t gexec = nullptr;
    int g_len = 0;
    double g_beta = -1.0;
    int g_kernel = -1;
    double kappa = 0.0;
    double yscale = 1.0;          // spread of the observed values (network input scale)
    void *ws_x = nullptr;         // network input buffer (allocated on first use)
    // the observations sorted by base cell on the device (x, y pairs, then values, then noise
    // variances; 4 m doubles), and a host copy made on first use: the multigrid levels are built
    // from it
    double *dsorted = nullptr;
    std::vector<double> hxy, hy, hvar;
    // prior mean (allocated on first use)
    double *fb = nullptr;         // n: prior mean f_b (NULL: zero)
    double *tgt64 = nullptr;      // n: cell-factor targets L f_b in FP64
    void *tgtT = nullptr;         // n: the targets in the message precision
    float2 *tgtdf = nullptr;      // n: the targets as double-float pairs (FP32 contexts)
};

namespace {

thread_local std::string t_create_err;
// set while a batch creates its members: rows of the message planes of odd-width problems are
// padded by one cell (DevProblem::px), so that the batched TMA kernel copies them as tensors
thread_local bool t_pad_odd_planes = false;

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

int fail(gabp_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(gabp_ctx *c, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();   // clear a non-sticky error
    return fail(c, e == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA, m);
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// Device memory of contexts comes from one stream-ordered pool per device, which keeps up to
// 8 GiB of freed memory for the next context: repeated create / destroy of a problem (a new
// analysis window on the same grid) reuses it instead of mapping and unmapping pages.
cudaMemPool_t context_pool(int dev) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0) return nullptr;
    if ((int)pools.size() <= dev) pools.resize((size_t)dev + 1, nullptr);
    if (!pools[(size_t)dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = (uint64_t)8 << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[(size_t)dev] = pool;
    }
    return pools[(size_t)dev];
}

int dalloc(gabp_ctx *c, void **ptr, size_t bytes, const char *what) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = context_pool(c->dev);
    cudaError_t e = pool ? cudaMallocFromPoolAsync(ptr, bytes, pool, c->stream) : cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    c->allocs.push_back({*ptr, pool != nullptr});
    return GABP_OK;
}

bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void drop_graph(gabp_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->g_len = 0;
    c->g_beta = -1.0;
    c->g_kernel = -1;
}

cudaError_t launch_iteration(gabp_ctx *c, int src, double beta, cudaStream_t st) {
    if (c->kernel == GABP_KERNEL_SPLIT) return gabp::launch_split_iteration(c->p, src, beta, st);
    if (c->kernel == GABP_KERNEL_TMA) return gabp::launch_tma_iteration(c->p, c->maps, src, beta, st);
    if (c->kernel == GABP_KERNEL_SWEEP) return gabp::launch_sweep_iteration(c->p, src, beta, c->shape.ty, st);
    if (c->p.order == 2) return gabp::launch_fused_l2_iteration(c->p, c->shape.ty, c->l2_run, src, beta, st);
    return gabp::launch_fused_iteration(c->p, src, beta, c->shape, st);
}

// A kernel's bounded wait gave up: report it (and clear the flag).
int check_device_error(gabp_ctx *c) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->p.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "error flag copy");
    CK(cudaStreamSynchronize(c->stream), "error flag sync");
    if (h) {
        CK(cudaMemsetAsync(c->p.err, 0, sizeof(int), c->stream), "error flag reset");
        CK(cudaStreamSynchronize(c->stream), "error flag sync");
        return fail(c, GABP_ERR_TIMEOUT, "a bounded wait inside the iteration kernel gave up");
    }
    return GABP_OK;
}

// Graph of `len` (even) iterations starting from buffer 0.
int ensure_graph(gabp_ctx *c, int len, double beta) {
    if (c->gexec && c->g_len == len && c->g_beta == beta && c->g_kernel == c->kernel) return GABP_OK;
    drop_graph(c);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t le = cudaSuccess;
    for (int t = 0; t < len && le == cudaSuccess; ++t) le = launch_iteration(c, t & 1, beta, c->cap);
    cudaError_t ee = cudaStreamEndCapture(c->cap, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, le, "iteration launch during capture");
    }
    if (ee != cudaSuccess) return cuda_fail(c, ee, "end capture");
    cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, ie, "graph instantiate");
    }
    c->g_len = len;
    c->g_beta = beta;
    c->g_kernel = c->kernel;
    return GABP_OK;
}

int run_iterations(gabp_ctx *c, int64_t count, double beta) {
    const int G = 20;
    if (count > 0 && c->cur == 1) {
        CK(launch_iteration(c, 1, beta, c->stream), "iteration launch");
        c->cur = 0;
        --count;
        ++c->iters;
    }
    if (count >= G) {
        int rc = ensure_graph(c, G, beta);
        if (rc != GABP_OK) return rc;
        while (count >= G) {
            CK(cudaGraphLaunch(c->gexec, c->stream), "graph launch");
            count -= G;
            c->iters += G;
        }
    }
    while (count > 0) {
        CK(launch_iteration(c, c->cur, beta, c->stream), "iteration launch");
        c->cur ^= 1;
        --count;
        ++c->iters;
    }
    return GABP_OK;
}

int compute_residual(gabp_ctx *c, double *out) {
    CK(gabp::launch_residual(c->p, c->cur, c->stream), "residual kernels");
    CK(cudaMemcpyAsync(c->hscal, c->p.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "residual copy");
    CK(cudaStreamSynchronize(c->stream), "residual sync");
    const double r2 = c->hscal[0], b2 = c->hscal[1];
    *out = b2 > 0.0 ? std::sqrt(r2) / std::sqrt(b2) : std::sqrt(r2);
    c->last_res = *out;
    return GABP_OK;
}

// mean over the 2 E message components (eta and Lambda of every factor-variable edge) of
// |m_t - m_{t-1}|, the quantity of the early-stopping rule (App. B)
int compute_msg_change(gabp_ctx *c, double *out) {
    CK(gabp::launch_msg_change(c->p, c->cur, c->p.scal + 2, c->stream), "message change kernels");
    CK(cudaMemcpyAsync(c->hscal + 2, c->p.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "message change copy");
    CK(cudaStreamSynchronize(c->stream), "message change sync");
    *out = c->hscal[2] / (2.0 * (double)c->edges);
    return GABP_OK;
}

size_t tsize(const gabp_ctx *c) { return c->p.prec ? sizeof(double) : sizeof(float); }

// Cell-factor targets r = L f_b of the prior mean (none without one).  The iteration kernels
// and the residual read them through the DevProblem, so the captured graph is dropped.
int set_targets(gabp_ctx *c) {
    gabp::DevProblem &p = c->p;
    if (c->fb) CK(gabp::launch_cell_targets(p, c->fb, c->tgt64, c->tgtT, c->tgtdf, c->stream), "prior targets");
    p.ptgt = c->fb ? c->tgtT : nullptr;
    p.ptgt64 = c->fb ? c->tgt64 : nullptr;
    p.ptgtdf = c->fb ? c->tgtdf : nullptr;
    drop_graph(c);
    return GABP_OK;
}

// Buffers of the prior mean (once per context).
int alloc_targets(gabp_ctx *c) {
    int rc;
    void *q;
    const int64_t n = c->p.n;
    if (!c->tgt64) {
        if ((rc = dalloc(c, &q, (size_t)n * sizeof(double), "alloc targets"))) return rc;
        c->tgt64 = (double *)q;
        if ((rc = dalloc(c, &c->tgtT, (size_t)n * tsize(c), "alloc targets"))) return rc;
        if (c->p.prec == 0) {
            if ((rc = dalloc(c, &q, (size_t)n * sizeof(float2), "alloc targets"))) return rc;
            c->tgtdf = (float2 *)q;
        }
    }
    return GABP_OK;
}

int init_messages(gabp_ctx *c) {
    CK(gabp::launch_init_cold(c->p, 0, c->opt.init == GABP_INIT_PAPER, c->stream), "init kernels");
    c->cur = 0;
    c->iters = 0;
    c->last_res = NAN;
    return GABP_OK;
}

void free_all(gabp_ctx *c) {
    drop_graph(c);
    if (c->ws_x) cudaFree(c->ws_x);
    c->ws_x = nullptr;
    for (const auto &a : c->allocs) {
        if (a.second) cudaFreeAsync(a.first, c->stream);
        else cudaFree(a.first);
    }
    if (!c->allocs.empty() && c->stream) cudaStreamSynchronize(c->stream);   // freed before reuse
    c->allocs.clear();
    if (c->hscal) cudaFreeHost(c->hscal);
    c->hscal = nullptr;
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    c->cap = nullptr;
    c->stream = nullptr;
}


// Host set-up work in parallel chunks: chunk ch of nchunk covers [ch * count / nchunk, ...); the
// results of every caller below do not depend on the number of chunks.
int host_chunks(int64_t count) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int64_t by_size = count / 65536 + 1;   // small inputs stay on one thread
    int64_t t = hw ? (int64_t)hw : 1;
    if (t > 32) t = 32;
    return (int)(t < by_size ? t : by_size);
}

// Host worker pool for the set-up chunks: up to hardware_concurrency - 1 threads, made on first
// use and kept for the process (detached, parked on a condition variable), so that a region
// costs a wake-up instead of a thread creation per chunk.  One region runs on the pool at a
// time; a region that finds it busy (another host thread's) spawns its own threads.
struct HostPool {
    std::mutex run_mu;   // held by the region using the pool
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::function<void(int)> job;   // runs chunk ch of the current region
    int nchunk = 0, next = 0, done = 0;
    int workers = 0;
};

HostPool *host_pool() {
    static HostPool *pool = new HostPool();   // never destroyed: its threads outlive static destruction
    return pool;
}

void host_pool_worker(HostPool *p) {
    std::unique_lock<std::mutex> lk(p->mu);
    for (;;) {
        p->cv_work.wait(lk, [p] { return p->next < p->nchunk; });
        const int ch = p->next++;
        lk.unlock();
        p->job(ch);
        lk.lock();
        if (++p->done == p->nchunk) p->cv_done.notify_one();
    }
}

template <typename F> void parallel_chunks(int64_t count, int nchunk, F f) {
    if (nchunk <= 1) {
        f(0, (int64_t)0, count);
        return;
    }
    auto chunk = [&](int ch) { f(ch, count * ch / nchunk, count * (ch + 1) / nchunk); };
    HostPool *p = host_pool();
    std::unique_lock<std::mutex> run(p->run_mu, std::try_to_lock);
    if (!run.owns_lock()) {
        std::vector<std::thread> th;
        th.reserve((size_t)nchunk - 1);
        for (int ch = 1; ch < nchunk; ++ch) th.emplace_back(chunk, ch);
        chunk(0);
        for (std::thread &t : th) t.join();
        return;
    }
    {
        std::lock_guard<std::mutex> lk(p->mu);
        while (p->workers < nchunk - 1) {
            std::thread(host_pool_worker, p).detach();
            ++p->workers;
        }
        p->job = chunk;
        p->done = 0;
        p->next = 0;
        p->nchunk = nchunk;
    }
    p->cv_work.notify_all();
    // this thread takes chunks too, then waits for the others
    std::unique_lock<std::mutex> lk(p->mu);
    while (p->next < p->nchunk) {
        const int ch = p->next++;
        lk.unlock();
        chunk(ch);
        lk.lock();
        ++p->done;
    }
    p->cv_done.wait(lk, [p] { return p->done == p->nchunk; });
    p->nchunk = 0;
    p->next = 0;
    p->job = nullptr;
}

int create_impl(gabp_ctx *c, gabp_grid grid, double kappa_h, const gabp_prior *prior, int64_t m,
                const double *obs_xy, const double *y, const double *noise_var) {
    const int nx = grid.nx, ny = grid.ny;
    if (nx < 1 || ny < 1) return fail(c, GABP_ERR_ARG, "grid sizes must be >= 1");
    if ((int64_t)nx * ny > (int64_t)1 << 30) return fail(c, GABP_ERR_ARG, "grid larger than 2^30 nodes");
    const double h = grid.h;
    if (!(h > 0.0) || !std::isfinite(h)) return fail(c, GABP_ERR_ARG, "grid spacing h must be finite and > 0");
    if (!(kappa_h > 0.0) || !std::isfinite(kappa_h)) return fail(c, GABP_ERR_ARG, "kappa must be finite and > 0");
    const double gamma_h = prior ? prior->gamma : 1.0;
    if (!(gamma_h > 0.0) || !std::isfinite(gamma_h)) return fail(c, GABP_ERR_ARG, "gamma must be finite and > 0");
    if (prior && prior->boundary != 0) return fail(c, GABP_ERR_ARG, "only the zero-Neumann boundary (0) is implemented");
    const int alpha = prior && prior->alpha ? prior->alpha : 2;
    if (alpha != 2 && alpha != 4) return fail(c, GABP_ERR_ARG, "alpha must be 2 or 4");
    // spacing h: L_h = kappa^2 I - Delta_h = h^-2 L_1(kappa h), so the prior gamma (L_h^(alpha/2))^T
    // L_h^(alpha/2) is the unit-spacing one with kappa h and gamma / h^(2 alpha); everything
    // below (kernels, multigrid, warm starts) works at unit spacing
    const double kappa = kappa_h * h;
    double hp = h * h;
    hp = hp * hp;
    if (alpha == 4) hp = hp * hp;
    const double gamma = gamma_h / hp;
    if (!(kappa > 0.0) || !std::isfinite(kappa) || !(gamma > 0.0) || !std::isfinite(gamma))
        return fail(c, GABP_ERR_ARG, "kappa h and gamma / h^(2 alpha) must be finite and > 0");
    if (m < 0 || m > ((int64_t)1 << 28)) return fail(c, GABP_ERR_ARG, "observation count out of range");
    if (m > 0 && (!obs_xy || !y || !noise_var)) return fail(c, GABP_ERR_ARG, "observation arrays must not be NULL");
    if (m > 0 && (nx < 2 || ny < 2)) return fail(c, GABP_ERR_ARG, "observations need a grid of at least 2 x 2");
    const gabp_options &o = c->opt;
    if (o.precision != GABP_FP32 && o.precision != GABP_FP64) return fail(c, GABP_ERR_ARG, "bad precision");
    if (o.init != GABP_INIT_COLD && o.init != GABP_INIT_PAPER) return fail(c, GABP_ERR_ARG, "bad init mode");
    if (o.kernel < GABP_KERNEL_AUTO || o.kernel > GABP_KERNEL_SWEEP) return fail(c, GABP_ERR_ARG, "bad kernel");
    if (!(o.tol > 0.0) || o.check_every < 1 || o.max_iters < 1) return fail(c, GABP_ERR_ARG, "bad tol/check_every/max_iters");
    if (o.tile_run < 0 || o.tile_run > 8) return fail(c, GABP_ERR_ARG, "tile_run must be 0..8");
    if (alpha == 4) {
        // FP32: the fused tile kernel (AUTO or FUSED, tiles 28 x 4 or 28 x 8) or the split kernels;
        // FP64: the split kernels
        if (o.kernel != GABP_KERNEL_AUTO && o.kernel != GABP_KERNEL_SPLIT && o.kernel != GABP_KERNEL_FUSED)
            return fail(c, GABP_ERR_ARG, "the alpha = 4 prior runs the fused or the split kernels");
        if (o.kernel == GABP_KERNEL_FUSED && o.precision != GABP_FP32)
            return fail(c, GABP_ERR_ARG, "the fused alpha = 4 kernel needs FP32 messages");
        const bool fused = o.precision == GABP_FP32 && o.kernel != GABP_KERNEL_SPLIT;
        if ((o.tile_x || o.tile_y) && !(fused && o.tile_x == 28 && gabp::fused_l2_shape_supported(o.tile_y)))
            return fail(c, GABP_ERR_ARG, "unsupported tile shape for the alpha = 4 prior (fused kernel: 28 x 4 or 28 x 8)");
    } else {
        // the kernel AUTO resolves to: the sweep for FP32, the plain fused kernel for FP64
        const int k = o.kernel != GABP_KERNEL_AUTO
                          ? o.kernel
                          : (o.precision == GABP_FP32 ? (nx % 4 == 0 && nx >= 4 ? GABP_KERNEL_TMA : GABP_KERNEL_SWEEP)
                                                      : GABP_KERNEL_FUSED);
        const bool tiled = o.tile_x || o.tile_y;
        if (tiled && (k == GABP_KERNEL_FUSED || k == GABP_KERNEL_SPLIT) && !gabp::fused_shape_supported(o.tile_x, o.tile_y))
            return fail(c, GABP_ERR_ARG, "unsupported tile shape");
        if (tiled && k == GABP_KERNEL_SWEEP && !(o.tile_x == 30 && gabp::sweep_shape_supported(o.tile_y)))
            return fail(c, GABP_ERR_ARG, "unsupported tile shape for the sweep kernel (30 x 16/32/64/128)");
        if (tiled && k == GABP_KERNEL_TMA && !gabp::tma_shape_supported(o.tile_x, o.tile_y))
            return fail(c, GABP_ERR_ARG, "unsupported tile shape for the TMA kernel");
    }
    const int64_t n = (int64_t)nx * ny;
    c->kappa = kappa;
    // host checks of the observations, run while the GPU copies and sorts them (below; those
    // kernels index nothing by the values, so invalid input cannot make them fault): validation
    // in parallel chunks, the first invalid index deciding the error, then the spread of y
    auto host_checks = [&]() -> int {
        const int nchunk = host_chunks(m);
        std::vector<int64_t> first_bad((size_t)nchunk, -1);
        std::vector<int> bad_kind((size_t)nchunk, 0);
        parallel_chunks(m, nchunk, [&](int ch, int64_t k0, int64_t k1) {
            for (int64_t k = k0; k < k1; ++k) {
                const double x = obs_xy[2 * k], yy = obs_xy[2 * k + 1];
                int kind = 0;
                if (!std::isfinite(x) || !std::isfinite(yy) || !std::isfinite(y[k]) || !std::isfinite(noise_var[k])) kind = 1;
                else if (x < 0.0 || x > nx - 1.0 || yy < 0.0 || yy > ny - 1.0) kind = 2;
                else if (!(noise_var[k] > 0.0)) kind = 3;
                if (kind) {
                    first_bad[(size_t)ch] = k;
                    bad_kind[(size_t)ch] = kind;
                    return;
                }
            }
        });
        for (int ch = 0; ch < nchunk; ++ch) {
            const int64_t k = first_bad[(size_t)ch];
            if (k < 0) continue;
            if (bad_kind[(size_t)ch] == 1) return fail(c, GABP_ERR_ARG, "non-finite observation data at index " + std::to_string(k));
            if (bad_kind[(size_t)ch] == 2) return fail(c, GABP_ERR_ARG, "observation " + std::to_string(k) + " outside the grid");
            return fail(c, GABP_ERR_ARG, "noise variance must be > 0");
        }
        if (m >= 2) {
            // sample standard deviation of y: partial sums over a fixed partition (64 parts,
            // whatever the thread count), added in part order
            constexpr int PARTS = 64;
            std::vector<double> part((size_t)PARTS);
            auto sum_parts = [&](auto term) {
                parallel_chunks(PARTS, host_chunks(m) > 1 ? (int)std::min<int64_t>(PARTS, host_chunks(m)) : 1,
                                [&](int, int64_t q0, int64_t q1) {
                                    for (int64_t q = q0; q < q1; ++q) {
                                        double acc = 0.0;
                                        for (int64_t k = m * q / PARTS; k < m * (q + 1) / PARTS; ++k) acc += term(k);
                                        part[(size_t)q] = acc;
                                    }
                                });
                double total = 0.0;
                for (double v : part) total += v;
                return total;
            };
            const double mean = sum_parts([&](int64_t k) { return y[k]; }) / (double)m;
            const double sq = sum_parts([&](int64_t k) { return (y[k] - mean) * (y[k] - mean); });
            const double sd = std::sqrt(sq / (double)(m - 1));
            c->yscale = sd > 0.0 ? sd : 1.0;
        }
        return GABP_OK;
    };
    DevProblem &p = c->p;
    p.nx = nx;
    p.px = (t_pad_odd_planes && nx % 2 && alpha == 2) ? nx + 1 : nx;
    p.pn = (int64_t)p.px * ny;
    p.ny = ny;
    p.n = n;
    p.m = m;
    p.prec = o.precision;
    p.gamma = gamma;
    p.debug_stall = (o.debug_flags & 1) ? 1 : 0;
    p.order = alpha == 4 ? 2 : 1;
    p.planes = alpha == 4 ? 13 : 5;
    for (int d = 0; d <= 4; ++d) p.aC[d] = kappa * kappa + (double)d;
    p.var_f = (float)(1.0 / gamma);
    for (int d = 0; d <= 4; ++d) {
        p.aC_f[d] = (float)p.aC[d];
        p.aC_lo[d] = (float)(p.aC[d] - (double)p.aC_f[d]);
    }
    p.gam_hi = (float)gamma;
    p.gam_lo = (float)(gamma - (double)p.gam_hi);
    for (int d = 0; d <= 4; ++d) p.init_c_f[d] = (float)(gamma * p.aC[d] * p.aC[d]);
    p.init_n_f = (float)(gamma * -1.0 * -1.0);
    for (int dc = 0; dc <= 4; ++dc) {   // alpha = 4 coefficients of FP32 contexts, rounded once
        p.l2c_f[dc] = (float)(p.aC[dc] * p.aC[dc] + (double)dc);
        for (int du = 0; du <= 4; ++du) p.l2n_f[5 * dc + du] = (float)(-(p.aC[dc] + p.aC[du]));
    }
    p.owdf = nullptr;
    p.oysdf = nullptr;
    const size_t T = tsize(c);
    int rc;
    void *q;
    for (int b = 0; b < 2; ++b) {
        if ((rc = dalloc(c, &p.P[b], (size_t)p.planes * (size_t)p.pn * 2 * T, "alloc prior messages"))) return rc;
        if ((rc = dalloc(c, &p.O[b], 8 * (size_t)m * T, "alloc obs messages"))) return rc;
        // padding cells: (0, 0) in both buffers, never written by a kernel
        if (p.px != nx)
            CK(cudaMemsetAsync(p.P[b], 0, (size_t)p.planes * (size_t)p.pn * 2 * T, c->stream), "memset planes");
    }
    if ((rc = dalloc(c, &q, (size_t)m * sizeof(int), "alloc obs base"))) return rc;
    p.obase = (const int *)q;
    if ((rc = dalloc(c, &q, 4 * (size_t)m * T, "alloc obs weights"))) return rc;
    p.ow = q;
    if ((rc = dalloc(c, &q, 2 * (size_t)m * T, "alloc obs values"))) return rc;
    p.ovar = q;
    if ((rc = dalloc(c, &q, 4 * (size_t)m * sizeof(double), "alloc obs weights fp64"))) return rc;
    p.ow64 = (const double *)q;
    if ((rc = dalloc(c, &q, 2 * (size_t)m * sizeof(double), "alloc obs values fp64"))) return rc;
    p.oys64 = (const double *)q;
    if (p.prec == 0) {   // double-float copies for the FP32 contexts' residual
        if ((rc = dalloc(c, &q, 4 * (size_t)m * sizeof(float2), "alloc obs weights double-float"))) return rc;
        p.owdf = (const float2 *)q;
        if ((rc = dalloc(c, &q, 2 * (size_t)m * sizeof(float2), "alloc obs values double-float"))) return rc;
        p.oysdf = (const float2 *)q;
    }
    if ((rc = dalloc(c, &q, ((size_t)n + 1) * sizeof(int), "alloc obs pointers"))) return rc;
    p.optr = (const int *)q;
    if ((rc = dalloc(c, &p.belief, (size_t)n * 4 * T, "alloc beliefs"))) return rc;
    if ((rc = dalloc(c, &q, (size_t)n * sizeof(double), "alloc residual scratch"))) return rc;
    p.mu64 = (double *)q;
    if ((rc = dalloc(c, &q, (size_t)n * sizeof(double), "alloc residual scratch"))) return rc;
    p.z64 = (double *)q;
    if ((rc = dalloc(c, &q, (size_t)m * sizeof(double), "alloc residual scratch"))) return rc;
    p.e64 = (double *)q;
    if ((rc = dalloc(c, &q, gabp::RES_BLOCKS * sizeof(double), "alloc partial sums"))) return rc;
    p.part = (double *)q;
    if ((rc = dalloc(c, &q, 4 * sizeof(double), "alloc scalars"))) return rc;   // |r|^2, |b|^2, message change
    p.scal = (double *)q;
    if ((rc = dalloc(c, &q, sizeof(int), "alloc error flag"))) return rc;
    p.err = (int *)q;
    CK(cudaMemsetAsync(p.err, 0, sizeof(int), c->stream), "memset");
    if ((rc = dalloc(c, &q, 2 * (size_t)n * sizeof(double), "alloc staging"))) return rc;
    c->stage = (double *)q;
    CK(cudaMallocHost((void **)&c->hscal, 4 * sizeof(double)), "alloc pinned scalars");
    CK(cudaMemsetAsync(p.scal, 0, 4 * sizeof(double), c->stream), "memset");

    // upload the caller's observations as they are, then on the GPU: base cells, the stable
    // sort by base cell (sorted raw data kept in c->dsorted: x, y pairs, values, variances),
    // FP64 precompute of weights and 1/sigma^2.  The raw copy and the sort's scratch go through
    // the staging buffer when it is large enough.
    if (m > 0) {
        if ((rc = dalloc(c, &q, 4 * (size_t)m * sizeof(double), "alloc sorted observations"))) return rc;
        c->dsorted = (double *)q;
        const size_t need = 4 * (size_t)m * sizeof(double) + gabp::obs_sort_scratch_bytes(m);
        double *raw = nullptr;
        const bool own_raw = need > 2 * (size_t)n * sizeof(double);
        if (own_raw) CK(cudaMalloc((void **)&raw, need), "alloc raw observations");
        else raw = c->stage;
        cudaError_t e = cudaMemcpyAsync(raw, obs_xy, 2 * (size_t)m * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(raw + 2 * m, y, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(raw + 3 * m, noise_var, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        double *sxy = c->dsorted, *sy = sxy + 2 * m, *svar = sxy + 3 * m;
        if (e == cudaSuccess)
            e = gabp::launch_obs_sort(m, nx, ny, raw, raw + 2 * m, raw + 3 * m, (int *)p.obase, sxy, sy, svar, raw + 4 * m,
                                      c->stream);
        if (e == cudaSuccess) e = gabp::launch_obs_precompute(p, sxy, sy, svar, c->stream);
        if (e == cudaSuccess && p.prec == 0) e = gabp::launch_df_precompute(p, c->stream);
        const int hrc = host_checks();
        // invalid observations: nothing more is launched; wait for the copies of the caller's
        // arrays before returning
        if ((hrc != GABP_OK || own_raw) && e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (own_raw) cudaFree(raw);
        if (hrc != GABP_OK) return hrc;
        if (e != cudaSuccess) return cuda_fail(c, e, "observation upload/sort/precompute");
    }
    CK(gabp::launch_obs_pointers(p, c->stream), "observation pointers");
    CK(gabp::launch_rhs_norm(p, c->stream), "rhs norm");
    if ((rc = init_messages(c))) return rc;
    CK(cudaStreamSynchronize(c->stream), "create sync");

    // iteration kernel and tile shape
    const bool tma_ok = gabp::tma_problem_supported(p);
    if (o.kernel == GABP_KERNEL_TMA && !tma_ok)
        return fail(c, GABP_ERR_ARG, "the TMA kernel needs FP32 messages and nx a multiple of 4");
    if (o.kernel == GABP_KERNEL_SWEEP && p.prec != 0)
        return fail(c, GABP_ERR_ARG, "the sweep kernel needs FP32 messages");
    if (p.order == 2) c->kernel = o.kernel == GABP_KERNEL_SPLIT || p.prec ? GABP_KERNEL_SPLIT : GABP_KERNEL_FUSED;
    else if (o.kernel == GABP_KERNEL_SPLIT) c->kernel = GABP_KERNEL_SPLIT;
    else if (o.kernel == GABP_KERNEL_TMA || (o.kernel == GABP_KERNEL_AUTO && tma_ok)) c->kernel = GABP_KERNEL_TMA;
    else if (o.kernel == GABP_KERNEL_SWEEP || (o.kernel == GABP_KERNEL_AUTO && p.prec == 0)) c->kernel = GABP_KERNEL_SWEEP;
    else c->kernel = GABP_KERNEL_FUSED;
    if (c->kernel == GABP_KERNEL_SWEEP) {
        c->shape = o.tile_y ? gabp::FusedShape{30, o.tile_y} : gabp::FusedShape{30, 64};
    } else if (c->kernel == GABP_KERNEL_TMA) {
        c->shape = o.tile_x ? gabp::FusedShape{o.tile_x, o.tile_y} : gabp::FusedShape{30, 14};
        CK(gabp::make_tma_maps(p, c->shape.tx, c->shape.ty, c->maps), "tensor map encode");
        c->maps.run = o.tile_run ? o.tile_run : gabp::tma_choose_run(p, c->shape.ty);
    } else if (p.order == 2) {
        c->shape = {0, 0};
        if (c->kernel == GABP_KERNEL_FUSED) {
            c->shape = {28, o.tile_y ? o.tile_y : 8};
            c->l2_run = o.tile_run ? o.tile_run : gabp::fused_l2_choose_run(p, c->shape.ty);
        }
    } else if (o.tile_x) {
        c->shape = {o.tile_x, o.tile_y};
    } else {
        c->shape = p.prec ? gabp::FusedShape{32, 8} : gabp::FusedShape{64, 16};
    }
    c->edges = 5 * n - 2 * (int64_t)(nx + ny) + 4 * m;
    if (p.order == 2) {   // 13-slot cell factors: count the slots whose node exists
        static const int dx[13] = {0, -1, 1, 0, 0, -1, 1, -1, 1, -2, 2, 0, 0};
        static const int dy[13] = {0, 0, 0, -1, 1, -1, -1, 1, 1, 0, 0, -2, 2};
        int64_t e = 0;
        for (int d = 0; d < 13; ++d)
            e += (int64_t)std::max(0, nx - std::abs(dx[d])) * std::max(0, ny - std::abs(dy[d]));
        c->edges = e + 4 * m;
    }
    const double ebytes = 4.0 * (double)T;    // (eta, Lambda) read + write per edge
    c->bytes_per_iter = ebytes * (double)c->edges + 5.0 * (double)T * (double)m;
    return GABP_OK;
}

}  // namespace

extern "C" {

void gabp_default_options(gabp_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = GABP_FP32;
    o->init = GABP_INIT_COLD;
    o->kernel = GABP_KERNEL_AUTO;
    o->tol = 1e-5;
    o->check_every = 50;
    o->max_iters = 200000;
    o->device = -1;
    o->stream = nullptr;
}

const char *gabp_create_error(void) { return t_create_err.c_str(); }

int gabp_create(gabp_ctx **out, gabp_grid grid, double kappa, const gabp_prior *prior, int64_t m,
                const double *obs_xy, const double *y, const double *noise_var, const gabp_options *opt) {
    NvtxRange nvtx_range("gabp_create");
    t_create_err.clear();
    if (!out) {
        t_create_err = "out must not be NULL";
        return GABP_ERR_ARG;
    }
    *out = nullptr;
    gabp_ctx *c = new (std::nothrow) gabp_ctx();
    if (!c) {
        t_create_err = "host allocation failed";
        return GABP_ERR_OOM;
    }
    if (opt) c->opt = *opt;
    else gabp_default_options(&c->opt);
    int dev = c->opt.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        t_create_err = "no CUDA device";
        delete c;
        return GABP_ERR_CUDA;
    }
    c->dev = dev;
    int rc = GABP_OK;
    {
        DeviceGuard g(dev);
        if (!g.ok) {
            rc = fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
        } else {
            cudaError_t e = cudaSuccess;
            if (c->opt.stream) {
                c->stream = (cudaStream_t)c->opt.stream;
            } else {
                e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
                c->own_stream = e == cudaSuccess;
            }
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) rc = cuda_fail(c, e, "stream create");
            else rc = create_impl(c, grid, kappa, prior, m, obs_xy, y, noise_var);
        }
        if (rc != GABP_OK) {
            t_create_err = c->err;
            free_all(c);
        }
    }
    if (rc != GABP_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return GABP_OK;
}

int gabp_iterate(gabp_ctx *c, int n_iters, double damping) {
    NvtxRange nvtx_range("gabp_iterate");
    if (!c) return GABP_ERR_ARG;
    if (!(damping >= 0.0 && damping < 1.0)) return fail(c, GABP_ERR_ARG, "damping must be in [0, 1)");
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    c->err.clear();
    if (n_iters >= 0) {
        const int cur0 = c->cur;
        const int64_t iters0 = c->iters;
        int rc = run_iterations(c, n_iters, damping);
        if (rc) return rc;
        CK(cudaStreamSynchronize(c->stream), "iterate sync");
        rc = check_device_error(c);
        if (rc) {   // a kernel gave up: point back at the messages the call started from
            c->cur = cur0;
            c->iters = iters0;
        }
        return rc;
    }
    double best = INFINITY, res = NAN;
    int64_t done = 0;
    for (;;) {
        int rc = compute_residual(c, &res);
        if (rc) return rc;
        if (!std::isfinite(res)) return fail(c, GABP_ERR_DIVERGED, "residual is not finite");
        if (res <= c->opt.tol) return GABP_OK;
        if (res > 1e6 * best) return fail(c, GABP_ERR_DIVERGED, "residual grew by more than 1e6");
        best = res < best ? res : best;
        if (done >= c->opt.max_iters)
            return fail(c, GABP_ERR_TIMEOUT, "max_iters reached with residual " + std::to_string(res));
        int64_t chunk = c->opt.check_every;
        if (done + chunk > c->opt.max_iters) chunk = c->opt.max_iters - done;
        rc = run_iterations(c, chunk, damping);
        if (rc) return rc;
        if ((rc = check_device_error(c))) return rc;
        done += chunk;
    }
}

int gabp_message_change(gabp_ctx *c, double *mean_abs_change) {
    if (!c || !mean_abs_change) return c ? fail(c, GABP_ERR_ARG, "mean_abs_change must not be NULL") : GABP_ERR_ARG;
    if (c->iters < 1) return fail(c, GABP_ERR_STATE, "no iteration since the last initialisation");
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    return compute_msg_change(c, mean_abs_change);
}

int gabp_iterate_early_stop(gabp_ctx *c, int max_iters, double damping, double tau, int check_every,
                            int64_t *stopped_at) {
    if (!c) return GABP_ERR_ARG;
    if (!(damping >= 0.0 && damping < 1.0)) return fail(c, GABP_ERR_ARG, "damping must be in [0, 1)");
    if (!(tau > 0.0) || check_every < 1 || max_iters < 3)
        return fail(c, GABP_ERR_ARG, "tau > 0, check_every >= 1 and max_iters >= 3 required");
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    c->err.clear();
    if (stopped_at) *stopped_at = 0;
    // iterations 1 and 2 of this call; the change of iteration 2 is the reference
    int rc = run_iterations(c, 2, damping);
    if (rc || (rc = check_device_error(c))) return rc;
    double ref = 0.0, d = 0.0;
    if ((rc = compute_msg_change(c, &ref))) return rc;
    if (!std::isfinite(ref)) return fail(c, GABP_ERR_DIVERGED, "message change is not finite");
    int64_t t = 2;
    for (;;) {
        if (t >= max_iters) return fail(c, GABP_ERR_TIMEOUT, "max_iters reached before the early-stopping rule held");
        int64_t chunk = check_every;
        if (t + chunk > max_iters) chunk = max_iters - t;
        rc = run_iterations(c, (int)chunk, damping);
        if (rc || (rc = check_device_error(c))) return rc;
        t += chunk;
        if ((rc = compute_msg_change(c, &d))) return rc;
        if (!std::isfinite(d)) return fail(c, GABP_ERR_DIVERGED, "message change is not finite");
        if (d < tau * ref) {
            if (stopped_at) *stopped_at = t;
            return GABP_OK;
        }
    }
}

int gabp_residual(gabp_ctx *c, double *rel) {
    NvtxRange nvtx_range("gabp_residual");
    if (!c || !rel) return c ? fail(c, GABP_ERR_ARG, "rel_residual must not be NULL") : GABP_ERR_ARG;
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    return compute_residual(c, rel);
}

int gabp_marginals(gabp_ctx *c, double *mean, double *var) {
    NvtxRange nvtx_range("gabp_marginals");
    if (!c) return GABP_ERR_ARG;
    if (!mean) return fail(c, GABP_ERR_ARG, "mean must not be NULL");
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    const int64_t n = c->p.n;
    // where the kernels write: device memory directly; pinned host memory through its device
    // address (the stores cross the host link while the kernel runs, no second pass); other host
    // memory through the staging buffer and a copy
    bool mapped = false;   // a kernel writes across the host link
    auto target = [&](double *ptr, double *stage, bool &copy) -> double * {
        copy = false;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
            cudaGetLastError();
            a.type = cudaMemoryTypeUnregistered;
        }
        if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return ptr;
        if (a.type == cudaMemoryTypeHost && a.devicePointer) {
            mapped = true;
            return static_cast<double *>(a.devicePointer);
        }
        copy = true;
        return stage;
    };
    bool cmean = false, cvar = false;
    double *kmean = target(mean, c->stage, cmean);
    double *kvar = var ? target(var, c->stage + n, cvar) : nullptr;
    CK(gabp::launch_marginals(c->p, c->cur, kmean, kvar, c->stream, !mapped), "marginal kernels");
    if (cmean) CK(cudaMemcpyAsync(mean, kmean, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy mean");
    if (cvar) CK(cudaMemcpyAsync(var, kvar, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy var");
    CK(cudaStreamSynchronize(c->stream), "marginals sync");
    return GABP_OK;
}

int gabp_warm_start(gabp_ctx *c, const double *mu0, const double *lam0) {
    NvtxRange nvtx_range("gabp_warm_start");
    if (!c) return GABP_ERR_ARG;
    if (c->p.order == 2) return fail(c, GABP_ERR_STATE, "warm starts are not available for the alpha = 4 prior");
    if (!mu0 || !lam0) return fail(c, GABP_ERR_ARG, "mu0 and lam0 must not be NULL");
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    const int64_t n = c->p.n;
    const double *dm = mu0, *dl = lam0;
    if (!is_device_ptr(mu0)) {
        CK(cudaMemcpyAsync(c->stage, mu0, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy mu0");
        dm = c->stage;
    }
    if (!is_device_ptr(lam0)) {
        CK(cudaMemcpyAsync(c->stage + n, lam0, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy lam0");
        dl = c->stage + n;
    }
    if (c->p.prec == 0) {
        // FP32 messages: FP32 arithmetic; the node pairs go to the staging buffer (each element
        // is read before its slot is written when mu0 itself was staged there)
        CK(gabp::launch_init_warm_f32(c->p, 0, dm, dl, (float2 *)c->stage, c->stream), "warm init kernels");
    } else {
        CK(gabp::launch_init_warm(c->p, 0, dm, dl, c->stream), "warm init kernels");
    }
    CK(cudaStreamSynchronize(c->stream), "warm start sync");
    c->cur = 0;
    c->iters = 0;
    c->last_res = NAN;
    return GABP_OK;
}

int gabp_reset(gabp_ctx *c) {
    if (!c) return GABP_ERR_ARG;
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    int rc = init_messages(c);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream), "reset sync");
    return GABP_OK;
}

int gabp_set_prior_mean(gabp_ctx *c, const double *f_b) {
    if (!c) return GABP_ERR_ARG;
    if (c->p.order == 2) return fail(c, GABP_ERR_STATE, "a prior mean is not available for the alpha = 4 prior");
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(c, GABP_ERR_CUDA, "cudaSetDevice failed");
    const int64_t n = c->p.n;
    int rc;
    if (f_b) {
        if ((rc = alloc_targets(c))) return rc;
        if (!c->fb) {
            void *q;
            if ((rc = dalloc(c, &q, (size_t)n * sizeof(double), "alloc prior mean"))) return rc;
            c->fb = (double *)q;
        }
        CK(cudaMemcpyAsync(c->fb, f_b, (size_t)n * sizeof(double), cudaMemcpyDefault, c->stream), "copy prior mean");
    } else {
        c->fb = nullptr;   // the buffer stays allocated with the context (freed at destroy)
    }
    if ((rc = set_targets(c))) return rc;
    CK(gabp::launch_rhs_norm(c->p, c->stream), "rhs norm");
    CK(cudaStreamSynchronize(c->stream), "prior mean sync");
    c->last_res = NAN;
    return GABP_OK;
}

int64_t gabp_message_bytes(const gabp_ctx *c) {
    if (!c) return -1;
    const int64_t T = c->p.prec ? 8 : 4;
    return 2 * (int64_t)c->p.planes * c->p.n * T + 8 * c->p.m * T;
}

int gabp_get_messages(gabp_ctx *c, void *buf) {
    if (!c || !buf) return c ? fail(c, GABP_ERR_ARG, "buffer must not be NULL") : GABP_ERR_ARG;
    if (c->p.px != c->p.nx) return fail(c, GABP_ERR_STATE, "padded message layout");   // batch members only
    DeviceGuard g(c->dev);
    const size_t T = tsize(c);
    const size_t pb = 2 * (size_t)c->p.planes * (size_t)c->p.n * T, ob = 8 * (size_t)c->p.m * T;
    CK(cudaMemcpyAsync(buf, c->p.P[c->cur], pb, cudaMemcpyDefault, c->stream), "copy messages");
    if (ob) CK(cudaMemcpyAsync((char *)buf + pb, c->p.O[c->cur], ob, cudaMemcpyDefault, c->stream), "copy messages");
    CK(cudaStreamSynchronize(c->stream), "messages sync");
    return GABP_OK;
}

int gabp_set_messages(gabp_ctx *c, const void *buf) {
    if (!c || !buf) return c ? fail(c, GABP_ERR_ARG, "buffer must not be NULL") : GABP_ERR_ARG;
    if (c->p.px != c->p.nx) return fail(c, GABP_ERR_STATE, "padded message layout");   // batch members only
    DeviceGuard g(c->dev);
    const size_t T = tsize(c);
    const size_t pb = 2 * (size_t)c->p.planes * (size_t)c->p.n * T, ob = 8 * (size_t)c->p.m * T;
    CK(cudaMemcpyAsync(c->p.P[0], buf, pb, cudaMemcpyDefault, c->stream), "copy messages");
    if (ob) CK(cudaMemcpyAsync(c->p.O[0], (const char *)buf + pb, ob, cudaMemcpyDefault, c->stream), "copy messages");
    CK(cudaStreamSynchronize(c->stream), "messages sync");
    c->cur = 0;
    return GABP_OK;
}

int gabp_get_stats(const gabp_ctx *c, gabp_stats *s) {
    if (!c || !s) return GABP_ERR_ARG;
    s->iterations = c->iters;
    s->last_residual = c->last_res;
    s->n = c->p.n;
    s->m = c->p.m;
    s->edges = c->edges;
    s->precision = c->p.prec;
    s->kernel = c->kernel;
    s->tile_x = c->shape.tx;
    s->tile_y = c->shape.ty;
    s->bytes_per_iter = c->bytes_per_iter;
    s->tile_run = c->kernel == GABP_KERNEL_TMA ? c->maps.run : c->p.order == 2 && c->kernel == GABP_KERNEL_FUSED ? c->l2_run : 0;
    return GABP_OK;
}

const char *gabp_last_error(const gabp_ctx *c) { return c ? c->err.c_str() : ""; }

void gabp_destroy(gabp_ctx *c) {
    if (!c) return;
    {
        DeviceGuard g(c->dev);
        if (c->stream) cudaStreamSynchronize(c->stream);
        free_all(c);
    }
    delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------------------

struct gabp_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap = nullptr;
    gabp_options opt{};
    std::vector<gabp_ctx *> inst;
    int kernel = GABP_KERNEL_SWEEP;   // GABP_KERNEL_TMA or GABP_KERNEL_SWEEP
    gabp::DevProblem *d_table = nullptr;
    int *d_prefix = nullptr;     // sweep: count + 1 strip offsets
    int *d_active = nullptr;     // sweep: count active flags
    int *h_active = nullptr;     // pinned: count active flags
    int *d_items = nullptr;      // TMA: [nitems, pad x 3, (problem, column, row, carry) x all_tiles]
    int *h_items = nullptr;      // pinned mirror
    int *d_err = nullptr;        // TMA: a bounded wait in the batched kernel gave up
    gabp::TmaMapsGlobal *d_maps = nullptr;   // TMA: the problems' tensor maps
    std::vector<int *> optr_pad;  // TMA: observation index with rows padded to a multiple of 4 ints
                                  // (problems whose nx is not one; nullptr otherwise)
    int all_tiles = 0;           // TMA: tiles of all problems at the current height (grid bound)
    int maps_ty = 0;             // TMA: tile height the tensor maps were encoded for
    double *h_scal = nullptr;    // pinned, 2 per problem
    int H = 64;
    int total_strips = 0;
    int cur = 0;
    std::vector<int64_t> iters;
    std::vector<double> res;
    std::string err;
    cudaGraphExec_t g_iter = nullptr;
    int g_len = 0;
    double g_beta = -1.0;
    int g_H = 0;
    cudaGraphExec_t g_res = nullptr;
};

namespace {

thread_local std::string t_batch_create_err;

int bfail(gabp_batch *b, int code, const std::string &msg) {
    if (b) b->err = msg;
    return code;
}

int bcuda(gabp_batch *b, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA, m);
}

#define BK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return bcuda(b, e_, what); \
    } while (0)

void batch_drop_graphs(gabp_batch *b) {
    if (b->g_iter) cudaGraphExecDestroy(b->g_iter);
    if (b->g_res) cudaGraphExecDestroy(b->g_res);
    b->g_iter = nullptr;
    b->g_res = nullptr;
    b->g_len = 0;
    b->g_beta = -1.0;
    b->g_H = 0;
}

int tma_tiles(const gabp::DevProblem &p, int ty) { return ((p.nx + 29) / 30) * ((p.ny + ty - 1) / ty); }

constexpr int TMA_MIN_TY = 14;   // the smallest batched TMA tile height (sizes the work-item list)

cudaError_t batch_launch(gabp_batch *b, int src, double beta, cudaStream_t st) {
    const int count = (int)b->inst.size();
    if (b->kernel == GABP_KERNEL_TMA) {
        gabp::TmaBatchArgs ba;
        ba.maps = b->d_maps;
        ba.table = b->d_table;
        ba.nitems = b->d_items;
        ba.items = reinterpret_cast<const int4 *>(b->d_items + 4);
        ba.err = b->d_err;
        ba.debug_stall = (b->opt.debug_flags & 1) ? 1 : 0;
        // the grid does not depend on the active set, so captured graphs stay valid when it changes
        return gabp::launch_tma_batch(ba, b->inst[0]->p, b->H, b->all_tiles, src, beta, st);
    }
    return gabp::launch_sweep_batch(b->d_table, b->d_prefix, b->d_active, count, b->total_strips, src, beta, b->H,
                                    st);
}

// Upload the active set (h_active[0 .. count)): flags for the sweep kernel; for the TMA kernel
// the (problem, tile) work items of the active problems.
// Work items of the active problems for the batched TMA kernel.  The tiles of every problem
// form runs of up to BATCH_RUN tiles down a tile column (bands of BATCH_RUN tile rows,
// band-major, problems in order); block b of the G blocks takes items b, b + G, ..., and each
// block, when its run is used up, takes the next run from the queue, so that most items sit
// directly below the same block's previous item (flag w = 1: two belief rows carry over).
// When the queue is empty a block takes the last tile of the longest remaining run.
constexpr int BATCH_RUN = 4;
int batch_upload_active(gabp_batch *b) {
    const int count = (int)b->inst.size();
    if (b->kernel == GABP_KERNEL_TMA) {
        const int G = gabp::tma_batch_grid(b->H, b->all_tiles);
        if (G < 1) return bfail(b, GABP_ERR_CUDA, "batched TMA kernel grid");
        struct Run {
            int prob, cx, cy, left;   // next tile (cx, cy), tiles left
        };
        std::vector<Run> runs;
        int64_t total = 0;
        for (int i = 0; i < count; ++i) {
            if (!b->h_active[i]) continue;
            const int ntx = (b->inst[i]->p.nx + 29) / 30, nty = (b->inst[i]->p.ny + b->H - 1) / b->H;
            for (int band = 0; band * BATCH_RUN < nty; ++band)
                for (int cx = 0; cx < ntx; ++cx)
                    runs.push_back({i, cx, band * BATCH_RUN, std::min(BATCH_RUN, nty - band * BATCH_RUN)});
            total += (int64_t)ntx * nty;
        }
        int4 *items = reinterpret_cast<int4 *>(b->h_items + 4);
        std::vector<Run> lane((size_t)G, Run{-1, 0, 0, 0});
        size_t next = 0;
        for (int64_t k = 0; k < total; ++k) {
            Run &r = lane[(size_t)(k % G)];
            int4 it;
            if (r.left == 0 && next < runs.size()) r = runs[next++];
            if (r.left > 0) {
                it = make_int4(r.prob, r.cx, r.cy, 0);
                ++r.cy;
                --r.left;
            } else {   // queue empty: the last tile of the longest remaining run
                size_t best = 0;
                for (size_t q = 1; q < lane.size(); ++q)
                    if (lane[q].left > lane[best].left) best = q;
                Run &o = lane[best];
                it = make_int4(o.prob, o.cx, o.cy + o.left - 1, 0);
                --o.left;
            }
            if (k >= G) {
                const int4 &pv = items[k - G];
                it.w = pv.x == it.x && pv.y == it.y && pv.z + 1 == it.z ? 1 : 0;
            }
            items[k] = it;
        }
        b->h_items[0] = (int)total;
        b->h_items[1] = b->h_items[2] = b->h_items[3] = 0;
        BK(cudaMemcpyAsync(b->d_items, b->h_items, sizeof(int) * (4 + 4 * (size_t)total), cudaMemcpyHostToDevice,
                           b->stream),
           "upload work items");
        return GABP_OK;
    }
    BK(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int) * count, cudaMemcpyHostToDevice, b->stream),
       "upload active flags");
    return GABP_OK;
}

// Tensor maps with boxes for 30 x ty tiles: the message planes of the problems with nx even
// (16-byte row strides; the batched TMA kernel copies the others with cp.async) and the
// observation index of every problem, from a copy whose rows are padded to a multiple of 4
// ints where nx is not one (made once, the index is fixed at creation).
int batch_encode_maps(gabp_batch *b, int ty) {
    const int count = (int)b->inst.size();
    std::vector<gabp::TmaMapsGlobal> maps(count);
    std::memset((void *)maps.data(), 0, sizeof(gabp::TmaMapsGlobal) * count);
    b->optr_pad.resize((size_t)count, nullptr);
    for (int i = 0; i < count; ++i) {
        const gabp::DevProblem &pi = b->inst[i]->p;
        const int nxi = pi.nx, pitch = (nxi + 3) & ~3;
        if (nxi % 4 != 0 && !b->optr_pad[i]) {
            BK(cudaMalloc((void **)&b->optr_pad[i], sizeof(int) * (size_t)pitch * pi.ny), "alloc padded index");
            BK(cudaMemcpy2DAsync(b->optr_pad[i], sizeof(int) * (size_t)pitch, pi.optr, sizeof(int) * (size_t)nxi,
                                 sizeof(int) * (size_t)nxi, pi.ny, cudaMemcpyDeviceToDevice, b->stream),
               "padded index copy");
        }
        const int parts = (pi.px % 2 == 0 ? gabp::TMA_MAP_PLANES : 0) | gabp::TMA_MAP_OPTR;
        gabp::TmaMaps m{};
        BK(gabp::make_tma_maps(pi, 30, ty, m, parts, b->optr_pad[i], pitch), "tensor map encode");
        maps[i].planes[0] = m.planes[0];
        maps[i].planes[1] = m.planes[1];
        maps[i].optr = m.optr;
    }
    BK(cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(gabp::TmaMapsGlobal) * count, cudaMemcpyHostToDevice,
                       b->stream),
       "upload tensor maps");
    BK(cudaStreamSynchronize(b->stream), "sync");   // the host copy of the maps goes out of scope
    b->maps_ty = ty;
    return GABP_OK;
}

// Kernel configuration of the batch: H = 22 or 30 selects the batched TMA kernel (30 x H tiles),
// 16, 32, 64 or 128 the sweep kernel with strips of H rows.  The active set is re-uploaded in the
// layout the kernel reads.
int batch_set_height(gabp_batch *b, int H) {
    const int count = (int)b->inst.size();
    if (gabp::tma_batch_shape_supported(H)) {
        b->kernel = GABP_KERNEL_TMA;
        if (b->maps_ty != H) {
            int rc = batch_encode_maps(b, H);
            if (rc) return rc;
        }
        b->all_tiles = 0;
        for (int i = 0; i < count; ++i) b->all_tiles += tma_tiles(b->inst[i]->p, H);
    } else {
        std::vector<int> pre(count + 1, 0);
        for (int i = 0; i < count; ++i)
            pre[i + 1] = pre[i] + gabp::sweep_strips(b->inst[i]->p.nx, b->inst[i]->p.ny, H);
        BK(cudaMemcpyAsync(b->d_prefix, pre.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, b->stream),
           "upload strip offsets");
        b->kernel = GABP_KERNEL_SWEEP;
        b->total_strips = pre[count];
    }
    b->H = H;
    int rc = batch_upload_active(b);
    if (rc) return rc;
    BK(cudaStreamSynchronize(b->stream), "sync");
    return GABP_OK;
}

// A bounded wait of the batched TMA kernel gave up: report it (and clear the flag).
int batch_check_error(gabp_batch *b) {
    if (b->kernel != GABP_KERNEL_TMA) return GABP_OK;
    int h = 0;
    BK(cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "error flag copy");
    BK(cudaStreamSynchronize(b->stream), "error flag sync");
    if (h) {
        BK(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "error flag reset");
        BK(cudaStreamSynchronize(b->stream), "error flag sync");
        return bfail(b, GABP_ERR_TIMEOUT, "a bounded wait inside the batched iteration kernel gave up");
    }
    return GABP_OK;
}

int batch_ensure_graph(gabp_batch *b, int len, double beta) {
    if (b->g_iter && b->g_len == len && b->g_beta == beta && b->g_H == b->H) return GABP_OK;
    if (b->g_iter) cudaGraphExecDestroy(b->g_iter);
    b->g_iter = nullptr;
    cudaGraph_t g = nullptr;
    BK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t le = cudaSuccess;
    for (int t = 0; t < len && le == cudaSuccess; ++t) le = batch_launch(b, t & 1, beta, b->cap);
    cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, le, "batch launch during capture");
    }
    if (ee != cudaSuccess) return bcuda(b, ee, "end capture");
    cudaError_t ie = cudaGraphInstantiate(&b->g_iter, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        b->g_iter = nullptr;
        return bcuda(b, ie, "graph instantiate");
    }
    b->g_len = len;
    b->g_beta = beta;
    b->g_H = b->H;
    return GABP_OK;
}

int batch_run(gabp_batch *b, int64_t count, double beta) {
    const int G = 20;
    if (count > 0 && b->cur == 1) {
        BK(batch_launch(b, 1, beta, b->stream), "batch launch");
        b->cur = 0;
        --count;
        for (size_t i = 0; i < b->inst.size(); ++i)
            if (b->h_active[i]) ++b->iters[i];
    }
    int64_t done = 0;
    if (count >= G) {
        int rc = batch_ensure_graph(b, G, beta);
        if (rc) return rc;
        while (count - done >= G) {
            BK(cudaGraphLaunch(b->g_iter, b->stream), "graph launch");
            done += G;
        }
    }
    while (done < count) {
        BK(batch_launch(b, b->cur, beta, b->stream), "batch launch");
        b->cur ^= 1;
        ++done;
    }
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (b->h_active[i]) b->iters[i] += count;
    for (gabp_ctx *c : b->inst) c->cur = b->cur;
    return GABP_OK;
}

// residuals of every problem at the current parity (graph captured per parity 0 only)
int batch_residuals(gabp_batch *b) {
    const int count = (int)b->inst.size();
    if (b->cur != 0 || !b->g_res) {
        if (b->g_res) cudaGraphExecDestroy(b->g_res);
        b->g_res = nullptr;
        cudaGraph_t g = nullptr;
        BK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t le = cudaSuccess;
        for (int i = 0; i < count && le == cudaSuccess; ++i) {
            le = gabp::launch_residual(b->inst[i]->p, b->cur, b->cap);
            if (le == cudaSuccess)
                le = cudaMemcpyAsync(b->h_scal + 2 * i, b->inst[i]->p.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                     b->cap);
        }
        cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bcuda(b, le, "residual capture");
        }
        if (ee != cudaSuccess) return bcuda(b, ee, "end capture");
        cudaError_t ie = cudaGraphInstantiate(&b->g_res, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            b->g_res = nullptr;
            return bcuda(b, ie, "graph instantiate");
        }
    }
    BK(cudaGraphLaunch(b->g_res, b->stream), "residual graph launch");
    BK(cudaStreamSynchronize(b->stream), "residual sync");
    if (int rc = batch_check_error(b)) return rc;
    if (b->cur != 0) {   // only the parity-0 graph is kept
        cudaGraphExecDestroy(b->g_res);
        b->g_res = nullptr;
    }
    for (int i = 0; i < count; ++i) {
        const double r2 = b->h_scal[2 * i], b2 = b->h_scal[2 * i + 1];
        b->res[i] = b2 > 0.0 ? std::sqrt(r2) / std::sqrt(b2) : std::sqrt(r2);
        b->inst[i]->last_res = b->res[i];
    }
    return GABP_OK;
}

std::string autotune_key(const gabp_batch *b) {
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, b->dev) == cudaSuccess ? prop.name : "unknown";
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    int64_t nodes = 0, obs = 0;
    for (const gabp_ctx *c : b->inst) {
        nodes += c->p.n;
        obs += c->p.m;
    }
    return "batch " + name + " " + std::to_string(b->inst.size()) + " " + std::to_string(nodes) + " " +
           std::to_string(obs);
}

int autotune_cache_lookup(const std::string &key) {
    const char *path = std::getenv("GABP_AUTOTUNE_CACHE");
    if (!path) return 0;
    FILE *f = std::fopen(path, "r");
    if (!f) return 0;
    char line[512];
    int found = 0;
    while (std::fgets(line, sizeof line, f)) {
        std::string s(line);
        const size_t sp = s.rfind(' ');
        if (sp != std::string::npos && s.compare(0, sp, key) == 0) found = std::atoi(s.c_str() + sp + 1);
    }
    std::fclose(f);
    return (gabp::tma_batch_shape_supported(found) || gabp::sweep_shape_supported(found)) ? found : 0;
}

void autotune_cache_store(const std::string &key, int value) {
    const char *path = std::getenv("GABP_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", key.c_str(), value);
    std::fclose(f);
}

// Time each candidate (the sweep kernel at each strip height, the batched TMA kernel at each tile
// height; `kernels` = GABP_KERNEL_AUTO for both, else the one kernel) on this batch and keep the
// fastest; messages are re-initialised afterwards.
int batch_autotune(gabp_batch *b, int kernels) {
    const std::string key = autotune_key(b) + " k" + std::to_string(kernels);
    int best = autotune_cache_lookup(key);
    if (!best) {
        std::vector<int> cands;
        if (kernels != GABP_KERNEL_TMA) cands.insert(cands.end(), {16, 32, 64, 128});
        if (kernels != GABP_KERNEL_SWEEP) cands.insert(cands.end(), {14, 22, 30});
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        BK(cudaEventCreate(&e0), "event");
        BK(cudaEventCreate(&e1), "event");
        for (int h : cands) {
            int rc = batch_set_height(b, h);
            if (rc) return rc;
            for (int t = 0; t < 2; ++t) BK(batch_launch(b, t & 1, 0.5, b->stream), "autotune launch");
            BK(cudaEventRecord(e0, b->stream), "event");
            for (int t = 0; t < 8; ++t) BK(batch_launch(b, t & 1, 0.5, b->stream), "autotune launch");
            BK(cudaEventRecord(e1, b->stream), "event");
            BK(cudaEventSynchronize(e1), "event sync");
            float ms = 0.f;
            BK(cudaEventElapsedTime(&ms, e0, e1), "event time");
            if (ms < best_ms) {
                best_ms = ms;
                best = h;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        autotune_cache_store(key, best);
    }
    int rc = batch_set_height(b, best);
    if (rc) return rc;
    for (gabp_ctx *c : b->inst) {
        rc = init_messages(c);
        if (rc) return bfail(b, rc, c->err);
    }
    BK(cudaStreamSynchronize(b->stream), "sync");
    b->cur = 0;
    return GABP_OK;
}

void batch_free(gabp_batch *b) {
    batch_drop_graphs(b);
    for (gabp_ctx *c : b->inst) gabp_destroy(c);
    b->inst.clear();
    if (b->d_table) cudaFree(b->d_table);
    if (b->d_prefix) cudaFree(b->d_prefix);
    if (b->d_active) cudaFree(b->d_active);
    if (b->d_err) cudaFree(b->d_err);
    if (b->d_items) cudaFree(b->d_items);
    if (b->h_items) cudaFreeHost(b->h_items);
    b->d_items = b->h_items = nullptr;
    if (b->d_maps) cudaFree(b->d_maps);
    for (int *q : b->optr_pad)
        if (q) cudaFree(q);
    b->optr_pad.clear();
    b->d_err = nullptr;
    b->d_maps = nullptr;
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->h_scal) cudaFreeHost(b->h_scal);
    b->d_table = nullptr;
    b->d_prefix = b->d_active = nullptr;
    b->h_active = nullptr;
    b->h_scal = nullptr;
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    b->cap = b->stream = nullptr;
}

int batch_create_impl(gabp_batch *b, int count, const gabp_problem *problems) {
    if (count < 1 || !problems) return bfail(b, GABP_ERR_ARG, "count must be >= 1 and problems non-NULL");
    if (b->opt.precision != GABP_FP32) return bfail(b, GABP_ERR_ARG, "batches use FP32 messages");
    const int kreq = b->opt.kernel, ty = b->opt.tile_y;
    if (kreq != GABP_KERNEL_AUTO && kreq != GABP_KERNEL_TMA && kreq != GABP_KERNEL_SWEEP)
        return bfail(b, GABP_ERR_ARG, "batches run the TMA or the sweep kernel");
    if (kreq == GABP_KERNEL_TMA && ty && !gabp::tma_batch_shape_supported(ty))
        return bfail(b, GABP_ERR_ARG, "the batched TMA kernel uses 30 x 14, 30 x 22 or 30 x 30 tiles");
    if (kreq == GABP_KERNEL_SWEEP && ty && !gabp::sweep_shape_supported(ty))
        return bfail(b, GABP_ERR_ARG, "strip height must be 16, 32, 64 or 128");
    if (kreq == GABP_KERNEL_AUTO && ty && !gabp::tma_batch_shape_supported(ty) && !gabp::sweep_shape_supported(ty))
        return bfail(b, GABP_ERR_ARG, "strip height must be 16, 32, 64 or 128 (sweep) or 14, 22, 30 (TMA)");
    gabp_options io = b->opt;
    io.stream = b->stream;
    io.kernel = GABP_KERNEL_SWEEP;
    io.tile_x = io.tile_y = 0;
    io.device = b->dev;
    for (int i = 0; i < count; ++i) {
        const gabp_problem &pr = problems[i];
        gabp_prior prior{pr.gamma > 0.0 ? pr.gamma : 1.0, 0, 2};
        gabp_ctx *c = nullptr;
        t_pad_odd_planes = true;
        const int rc = gabp_create(&c, pr.grid, pr.kappa, &prior, pr.m, pr.obs_xy, pr.y, pr.noise_var, &io);
        t_pad_odd_planes = false;
        if (rc) return bfail(b, rc, "problem " + std::to_string(i) + ": " + gabp_create_error());
        b->inst.push_back(c);
    }
    BK(cudaMalloc((void **)&b->d_table, sizeof(gabp::DevProblem) * count), "alloc table");
    BK(cudaMalloc((void **)&b->d_prefix, sizeof(int) * (count + 1)), "alloc strip offsets");
    BK(cudaMalloc((void **)&b->d_active, sizeof(int) * count), "alloc active flags");
    BK(cudaMallocHost((void **)&b->h_active, sizeof(int) * count), "alloc pinned flags");
    BK(cudaMallocHost((void **)&b->h_scal, 2 * sizeof(double) * count), "alloc pinned scalars");
    std::vector<gabp::DevProblem> table(count);
    for (int i = 0; i < count; ++i) {
        table[i] = b->inst[i]->p;
        b->h_active[i] = 1;
    }
    BK(cudaMemcpyAsync(b->d_table, table.data(), sizeof(gabp::DevProblem) * count, cudaMemcpyHostToDevice, b->stream),
       "upload table");
    int max_tiles = 0;
    for (int i = 0; i < count; ++i) max_tiles += tma_tiles(b->inst[i]->p, TMA_MIN_TY);
    BK(cudaMalloc((void **)&b->d_maps, sizeof(gabp::TmaMapsGlobal) * count), "alloc tensor maps");
    BK(cudaMalloc((void **)&b->d_items, sizeof(int) * (4 + 4 * (size_t)max_tiles)), "alloc work items");
    BK(cudaMallocHost((void **)&b->h_items, sizeof(int) * (4 + 4 * (size_t)max_tiles)), "alloc pinned items");
    BK(cudaMalloc((void **)&b->d_err, sizeof(int)), "alloc error flag");
    BK(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "memset");
    b->iters.assign(count, 0);
    b->res.assign(count, NAN);
    if (b->opt.check_every & 1) b->opt.check_every += 1;
    if (ty) return batch_set_height(b, ty);
    return batch_autotune(b, kreq);
}

}  // namespace

extern "C" {

int gabp_batch_create(gabp_batch **out, int count, const gabp_problem *problems, const gabp_options *opt) {
    t_batch_create_err.clear();
    if (!out) {
        t_batch_create_err = "out must not be NULL";
        return GABP_ERR_ARG;
    }
    *out = nullptr;
    gabp_batch *b = new (std::nothrow) gabp_batch();
    if (!b) return GABP_ERR_OOM;
    if (opt) b->opt = *opt;
    else gabp_default_options(&b->opt);
    int dev = b->opt.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        t_batch_create_err = "no CUDA device";
        return GABP_ERR_CUDA;
    }
    b->dev = dev;
    int rc = GABP_OK;
    {
        DeviceGuard g(dev);
        cudaError_t e = cudaSuccess;
        if (b->opt.stream) {
            b->stream = (cudaStream_t)b->opt.stream;
        } else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = e == cudaSuccess;
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        rc = (!g.ok || e != cudaSuccess) ? bcuda(b, e, "stream create") : batch_create_impl(b, count, problems);
        if (rc) {
            t_batch_create_err = b->err;
            batch_free(b);
        }
    }
    if (rc) {
        delete b;
        return rc;
    }
    *out = b;
    return GABP_OK;
}

int gabp_batch_iterate(gabp_batch *b, int n_iters, double damping) {
    NvtxRange nvtx_range("gabp_batch_iterate");
    if (!b) return GABP_ERR_ARG;
    if (!(damping >= 0.0 && damping < 1.0)) return bfail(b, GABP_ERR_ARG, "damping must be in [0, 1)");
    DeviceGuard g(b->dev);
    b->err.clear();
    const int count = (int)b->inst.size();
    if (n_iters >= 0) {
        for (int i = 0; i < count; ++i) b->h_active[i] = 1;
        int rc = batch_upload_active(b);
        if (rc) return rc;
        rc = batch_run(b, n_iters, damping);
        if (rc) return rc;
        BK(cudaStreamSynchronize(b->stream), "iterate sync");
        return batch_check_error(b);
    }
    int rc;
    if (b->cur == 1) {   // checks run at parity 0
        for (int i = 0; i < count; ++i) b->h_active[i] = 1;
        if ((rc = batch_upload_active(b))) return rc;
        if ((rc = batch_run(b, 1, damping))) return rc;
    }
    int64_t done = 0;
    for (;;) {
        if ((rc = batch_residuals(b))) return rc;
        int active = 0;
        for (int i = 0; i < count; ++i) {
            if (!std::isfinite(b->res[i]))
                return bfail(b, GABP_ERR_DIVERGED, "problem " + std::to_string(i) + ": residual is not finite");
            b->h_active[i] = b->res[i] > b->opt.tol ? 1 : 0;
            active += b->h_active[i];
        }
        if (!active) return GABP_OK;
        if (done >= b->opt.max_iters) return bfail(b, GABP_ERR_TIMEOUT, std::to_string(active) + " problems above tol at max_iters");
        if ((rc = batch_upload_active(b))) return rc;
        if ((rc = batch_run(b, b->opt.check_every, damping))) return rc;
        done += b->opt.check_every;
    }
}

int gabp_batch_residuals(gabp_batch *b, double *rel) {
    if (!b || !rel) return b ? bfail(b, GABP_ERR_ARG, "rel must not be NULL") : GABP_ERR_ARG;
    DeviceGuard g(b->dev);
    int rc = batch_residuals(b);
    if (rc) return rc;
    for (size_t i = 0; i < b->inst.size(); ++i) rel[i] = b->res[i];
    return GABP_OK;
}

int gabp_batch_marginals(gabp_batch *b, int index, double *mean, double *var) {
    if (!b) return GABP_ERR_ARG;
    if (index < 0 || index >= (int)b->inst.size()) return bfail(b, GABP_ERR_ARG, "index out of range");
    gabp_ctx *c = b->inst[index];
    c->cur = b->cur;
    const int rc = gabp_marginals(c, mean, var);
    if (rc) return bfail(b, rc, c->err);
    return GABP_OK;
}

int gabp_batch_get_stats(const gabp_batch *b, int index, gabp_stats *s) {
    if (!b || !s || index < 0 || index >= (int)b->inst.size()) return GABP_ERR_ARG;
    const int rc = gabp_get_stats(b->inst[index], s);
    s->iterations = b->iters[index];
    s->last_residual = b->res[index];
    s->kernel = b->kernel;
    s->tile_x = 30;
    s->tile_y = b->H;
    return rc;
}

int gabp_batch_strip_height(const gabp_batch *b) { return b ? b->H : 0; }

const char *gabp_batch_last_error(const gabp_batch *b) { return b ? b->err.c_str() : t_batch_create_err.c_str(); }

void gabp_batch_destroy(gabp_batch *b) {
    if (!b) return;
    {
        DeviceGuard g(b->dev);
        if (b->stream) cudaStreamSynchronize(b->stream);
        batch_free(b);
    }
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Learned warm start glue
// ---------------------------------------------------------------------------------------

namespace {

inline int pad8(int v) { return (v + 7) / 8 * 8; }

int ws_ensure_input(gabp_ctx *c) {
    if (c->ws_x) return GABP_OK;
    const size_t bytes = sizeof(uint16_t) * 16 * (size_t)pad8(c->p.nx) * pad8(c->p.ny);
    CK(cudaMalloc(&c->ws_x, bytes), "alloc network input");
    return GABP_OK;
}

int ws_sample(gabp_ctx *c, void *x_out, float *t_out) {
    const int Hp = pad8(c->p.ny), Wp = pad8(c->p.nx);
    if (x_out) CK(gabp::launch_ws_input(c->p, c->yscale, c->kappa, Hp, Wp, x_out, c->stream), "network input");
    if (t_out) CK(gabp::launch_ws_target(c->p, c->cur, c->yscale, Hp, Wp, t_out, c->stream), "network target");
    CK(cudaStreamSynchronize(c->stream), "sync");
    return GABP_OK;
}

}  // namespace

extern "C" {

int gabp_wsnet_input_shape(const gabp_ctx *c, int *H, int *W, double *scale) {
    if (!c) return GABP_ERR_ARG;
    if (H) *H = pad8(c->p.ny);
    if (W) *W = pad8(c->p.nx);
    if (scale) *scale = c->yscale;
    return GABP_OK;
}

int gabp_wsnet_sample(gabp_ctx *c, void *x_out, float *t_out) {
    if (!c) return GABP_ERR_ARG;
    DeviceGuard g(c->dev);
    return ws_sample(c, x_out, t_out);
}

int gabp_batch_wsnet_sample(gabp_batch *b, int index, void *x_out, float *t_out) {
    if (!b) return GABP_ERR_ARG;
    if (index < 0 || index >= (int)b->inst.size()) return bfail(b, GABP_ERR_ARG, "index out of range");
    DeviceGuard g(b->dev);
    gabp_ctx *c = b->inst[index];
    c->cur = b->cur;
    const int rc = ws_sample(c, x_out, t_out);
    if (rc) return bfail(b, rc, c->err);
    return GABP_OK;
}

int gabp_batch_input_shape(const gabp_batch *b, int index, int *H, int *W, double *scale) {
    if (!b || index < 0 || index >= (int)b->inst.size()) return GABP_ERR_ARG;
    return gabp_wsnet_input_shape(b->inst[index], H, W, scale);
}

// ---- multigrid warm start (Sec. 3.2 "Multigrid"; Alg. 2 "Multigrid MP", "Upscale Messages") ----
}  // extern "C"

struct gabp_mg {
    gabp_ctx *target = nullptr;
    int levels = 0;
    std::vector<gabp_ctx *> lv;   // lv[k] = level k (k >= 1); lv[0] unused (the target)
    double *mu[2] = {nullptr, nullptr}, *q[2] = {nullptr, nullptr};   // marginal buffers (target size)
    std::string err;
};

namespace {

int mfail(gabp_mg *g, int code, const std::string &msg) {
    g->err = msg;
    return code;
}

#define CK_MG(call, what)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return mfail(g, GABP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_));     \
        }                                                                                          \
    } while (0)

void mg_free(gabp_mg *g) {
    for (gabp_ctx *c : g->lv)
        if (c) gabp_destroy(c);
    g->lv.clear();
    for (int i = 0; i < 2; ++i) {
        if (g->mu[i]) cudaFree(g->mu[i]);
        if (g->q[i]) cudaFree(g->q[i]);
        g->mu[i] = g->q[i] = nullptr;
    }
}

// run one level: exactly max_iters iterations (tol <= 0) or until the relative residual is
// <= tol (checked every check_every iterations, at most max_iters); returns the final residual
int mg_run_level(gabp_ctx *c, double damping, double tol, int max_iters, double *res) {
    int rc;
    if (tol > 0.0) {
        c->opt.tol = tol;
        c->opt.max_iters = max_iters;
        rc = gabp_iterate(c, -1, damping);
        if (rc == GABP_ERR_TIMEOUT || rc == GABP_ERR_DIVERGED) rc = GABP_OK;   // decided by the residual
    } else {
        rc = gabp_iterate(c, max_iters, damping);
    }
    if (rc) return rc;
    return gabp_residual(c, res);
}

}  // namespace

extern "C" {

int gabp_mg_create(gabp_mg **out, gabp_ctx *ctx, int levels) {
    if (!out || !ctx) return GABP_ERR_ARG;
    *out = nullptr;
    if (levels < 2 || levels > GABP_MG_MAX_LEVELS) return fail(ctx, GABP_ERR_ARG, "levels must be in [2, 16]");
    if (ctx->p.order == 2) return fail(ctx, GABP_ERR_STATE, "multigrid is not available for the alpha = 4 prior");
    if (ctx->fb) return fail(ctx, GABP_ERR_STATE, "multigrid levels are built for a zero prior mean");
    const int nx = ctx->p.nx, ny = ctx->p.ny;
    const int64_t m = ctx->p.m;
    for (int k = 1; k < levels; ++k) {
        const int s = 1 << k;
        const int nxk = (nx + s - 1) / s, nyk = (ny + s - 1) / s;
        if (nxk < 2 || nyk < 2)
            return fail(ctx, GABP_ERR_ARG, "too many levels: level " + std::to_string(k) + " has fewer than 2 nodes per axis");
    }
    gabp_mg *g = new (std::nothrow) gabp_mg();
    if (!g) return GABP_ERR_OOM;
    g->target = ctx;
    g->levels = levels;
    g->lv.assign((size_t)levels, nullptr);
    DeviceGuard dg(ctx->dev);
    if (m > 0 && ctx->hxy.empty()) {   // host copy of the sorted observations, once
        std::vector<double> h(4 * (size_t)m);
        if (cudaMemcpyAsync(h.data(), ctx->dsorted, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            delete g;
            return fail(ctx, GABP_ERR_CUDA, "multigrid: observation download");
        }
        ctx->hxy.assign(h.begin(), h.begin() + 2 * m);
        ctx->hy.assign(h.begin() + 2 * m, h.begin() + 3 * m);
        ctx->hvar.assign(h.begin() + 3 * m, h.end());
    }
    std::vector<double> xy((size_t)(2 * m));
    int rc = GABP_OK;
    for (int k = 1; k < levels && rc == GABP_OK; ++k) {
        // level k: the same SPDE at spacing 2^k (kappa 2^k kappa, gamma / 4^k), every observation at
        // its coordinates on that grid, clamped to the last node
        const int s = 1 << k;
        const int nxk = (nx + s - 1) / s, nyk = (ny + s - 1) / s;
        for (int64_t i = 0; i < m; ++i) {
            xy[2 * i] = std::min(ctx->hxy[2 * i] / s, (double)(nxk - 1));
            xy[2 * i + 1] = std::min(ctx->hxy[2 * i + 1] / s, (double)(nyk - 1));
        }
        gabp_grid gk{nxk, nyk, 1.0};
        gabp_prior pk{ctx->p.gamma / ((double)s * s), 0, 2};
        gabp_options ok = ctx->opt;
        ok.kernel = GABP_KERNEL_AUTO;
        ok.tile_x = ok.tile_y = 0;
        ok.debug_flags = 0;
        ok.device = ctx->dev;
        ok.stream = ctx->stream;
        rc = gabp_create(&g->lv[(size_t)k], gk, ctx->kappa * s, &pk, m, xy.data(), ctx->hy.data(), ctx->hvar.data(), &ok);
        if (rc) fail(ctx, rc, "multigrid level " + std::to_string(k) + ": " + gabp_create_error());
    }
    for (int i = 0; i < 2 && rc == GABP_OK; ++i) {
        const size_t bytes = (size_t)ctx->p.n * sizeof(double);
        if (cudaMalloc((void **)&g->mu[i], bytes) != cudaSuccess || cudaMalloc((void **)&g->q[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(ctx, GABP_ERR_OOM, "multigrid buffers");
        }
    }
    if (rc) {
        mg_free(g);
        delete g;
        return rc;
    }
    *out = g;
    return GABP_OK;
}

int gabp_mg_warm_start(gabp_mg *g, double damping, double tol, int max_iters, gabp_mg_stats *stats) {
    NvtxRange nvtx_range("gabp_mg_warm_start");
    if (!g) return GABP_ERR_ARG;
    if (!(damping >= 0.0 && damping < 1.0)) return mfail(g, GABP_ERR_ARG, "damping must be in [0, 1)");
    if (max_iters < 1) return mfail(g, GABP_ERR_ARG, "max_iters must be >= 1");
    gabp_ctx *t = g->target;
    DeviceGuard dg(t->dev);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->levels = g->levels;
    }
    // (mu[cur], q[cur]): marginals handed to the next finer level, on the grid of level `have_k`
    int cur = 0, have_k = -1;
    for (int k = g->levels - 1; k >= 1; --k) {
        gabp_ctx *c = g->lv[(size_t)k];
        const int nxk = c->p.nx, nyk = c->p.ny;
        // this level's start: the upscaled state of level k+1 (precisions), or cold
        const bool warm = have_k == k + 1;
        if (warm) {
            gabp_ctx *u = g->lv[(size_t)k + 1];
            CK_MG(gabp::launch_upscale(g->mu[cur], g->q[cur], 0, 1, u->p.nx, u->p.ny, nxk, nyk, g->mu[cur ^ 1],
                                       g->q[cur ^ 1], c->stream),
                  "upscale");
            cur ^= 1;
        }
        // GaBP on this level; a run whose final relative residual is not finite or not below 1
        // is repeated from the same start with the damping (1 + b) / 2, up to three times
        double b = damping, used = damping, res = NAN;
        bool ok = false;
        int64_t its = 0;
        for (int attempt = 0; attempt <= 3 && !ok; ++attempt) {
            int rc = warm ? gabp_warm_start(c, g->mu[cur], g->q[cur]) : gabp_reset(c);
            if (rc) return mfail(g, rc, "multigrid level " + std::to_string(k) + ": " + c->err);
            used = b;
            rc = mg_run_level(c, b, tol, max_iters, &res);
            its += c->iters;
            if (rc) return mfail(g, rc, "multigrid level " + std::to_string(k) + ": " + c->err);
            ok = std::isfinite(res) && res < 1.0;
            b = 0.5 * (1.0 + b);
        }
        if (stats) {
            stats->iterations[k] = its;
            stats->damping[k] = used;
            stats->residual[k] = res;
            stats->converged[k] = ok ? 1 : 0;
        }
        if (ok) {
            // this level's marginals (mean, variance) into the other buffer pair
            const int o = cur ^ 1;
            int rc = gabp_marginals(c, g->mu[o], g->q[o]);
            if (rc) return mfail(g, rc, "multigrid level " + std::to_string(k) + ": " + c->err);
            CK_MG(gabp::launch_upscale(g->mu[o], g->q[o], 1, 0, nxk, nyk, nxk, nyk, g->mu[cur], g->q[cur], c->stream),
                  "precisions");
            have_k = k;
        } else if (warm) {
            have_k = k;   // pass this level's own start on (already in mu[cur], q[cur])
        }
    }
    // the target grid
    int rc;
    if (have_k == 1) {
        gabp_ctx *u = g->lv[1];
        CK_MG(gabp::launch_upscale(g->mu[cur], g->q[cur], 0, 1, u->p.nx, u->p.ny, t->p.nx, t->p.ny, g->mu[cur ^ 1],
                                   g->q[cur ^ 1], t->stream),
              "upscale");
        cur ^= 1;
        rc = gabp_warm_start(t, g->mu[cur], g->q[cur]);
    } else {
        rc = gabp_reset(t);
    }
    if (rc) return mfail(g, rc, std::string("target: ") + t->err);
    return GABP_OK;
}

const char *gabp_mg_last_error(const gabp_mg *g) { return g ? g->err.c_str() : ""; }

void gabp_mg_destroy(gabp_mg *g) {
    if (!g) return;
    DeviceGuard dg(g->target->dev);
    mg_free(g);
    delete g;
}

// ---- the paper's pairwise re-weighted form (App. A) ----
}  // extern "C"

struct gabp_pw {
    gabp_ctx *ctx = nullptr;
    void *Pd = nullptr, *hv = nullptr, *Pn = nullptr, *msg[2] = {nullptr, nullptr};
    int cur = 0;
    double c = 1.0;
    int64_t iters = 0;
    std::string err;
};

namespace {

int pfail(gabp_pw *w, int code, const std::string &msg) {
    w->err = msg;
    return code;
}

#define CK_PW(call, what)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return pfail(w, GABP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_));     \
        }                                                                                          \
    } while (0)

void pw_free(gabp_pw *w) {
    void *ps[5] = {w->Pd, w->hv, w->Pn, w->msg[0], w->msg[1]};
    for (void *q : ps)
        if (q) cudaFree(q);
    w->Pd = w->hv = w->Pn = w->msg[0] = w->msg[1] = nullptr;
}

}  // namespace

extern "C" {

int gabp_pw_create(gabp_pw **out, gabp_ctx *ctx) {
    if (!out || !ctx) return GABP_ERR_ARG;
    *out = nullptr;
    if (ctx->p.order == 2) return fail(ctx, GABP_ERR_STATE, "the pairwise form is built for the alpha = 2 prior only");
    if (ctx->fb) return fail(ctx, GABP_ERR_STATE, "the pairwise form is built for a zero prior mean");
    gabp_pw *w = new (std::nothrow) gabp_pw();
    if (!w) return GABP_ERR_OOM;
    w->ctx = ctx;
    DeviceGuard dg(ctx->dev);
    const size_t T = ctx->p.prec ? sizeof(double) : sizeof(float);
    const size_t n = (size_t)ctx->p.n;
    cudaError_t e = cudaMalloc(&w->Pd, n * T);
    if (e == cudaSuccess) e = cudaMalloc(&w->hv, n * T);
    if (e == cudaSuccess) e = cudaMalloc(&w->Pn, 12 * n * T);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&w->msg[b], 24 * n * T);
    if (e == cudaSuccess) e = gabp::pw_setup(ctx->p, w->Pd, w->hv, w->Pn, ctx->stream);
    if (e == cudaSuccess) e = gabp::pw_zero(ctx->p, w->msg[0], ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const int code = e == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA;
        fail(ctx, code, std::string("pairwise setup: ") + cudaGetErrorString(e));
        pw_free(w);
        delete w;
        return code;
    }
    *out = w;
    return GABP_OK;
}

int gabp_pw_iterate(gabp_pw *w, int n_iters, double c, double learning_rate) {
    NvtxRange nvtx_range("gabp_pw_iterate");
    if (!w) return GABP_ERR_ARG;
    if (n_iters < 0 || c == 0.0 || !std::isfinite(c) || !(learning_rate > 0.0 && learning_rate <= 1.0))
        return pfail(w, GABP_ERR_ARG, "n_iters >= 0, c finite and nonzero, learning_rate in (0, 1] required");
    gabp_ctx *ctx = w->ctx;
    DeviceGuard dg(ctx->dev);
    for (int t = 0; t < n_iters; ++t) {
        CK_PW(gabp::pw_iterate(ctx->p, w->Pd, w->hv, w->Pn, w->msg[w->cur], w->msg[w->cur ^ 1], c, learning_rate,
                               ctx->stream),
              "pairwise iteration");
        w->cur ^= 1;
    }
    CK_PW(cudaStreamSynchronize(ctx->stream), "pairwise sync");
    w->c = c;
    w->iters += n_iters;
    return GABP_OK;
}

int gabp_pw_marginals(gabp_pw *w, double *mean, double *var) {
    if (!w || !mean) return w ? pfail(w, GABP_ERR_ARG, "mean must not be NULL") : GABP_ERR_ARG;
    gabp_ctx *ctx = w->ctx;
    DeviceGuard dg(ctx->dev);
    const int64_t n = ctx->p.n;
    const bool dmean = is_device_ptr(mean), dvar = var ? is_device_ptr(var) : true;
    double *km = dmean ? mean : ctx->stage;
    double *kv = var ? (dvar ? var : ctx->stage + n) : nullptr;
    CK_PW(gabp::pw_marginals(ctx->p, w->Pd, w->hv, w->msg[w->cur], w->c, km, kv, 0, ctx->stream), "pairwise marginals");
    if (!dmean) CK_PW(cudaMemcpyAsync(mean, km, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy mean");
    if (var && !dvar) CK_PW(cudaMemcpyAsync(var, kv, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy var");
    CK_PW(cudaStreamSynchronize(ctx->stream), "pairwise marginals sync");
    return GABP_OK;
}

int gabp_pw_residual(gabp_pw *w, double *rel) {
    if (!w || !rel) return w ? pfail(w, GABP_ERR_ARG, "rel must not be NULL") : GABP_ERR_ARG;
    gabp_ctx *ctx = w->ctx;
    DeviceGuard dg(ctx->dev);
    CK_PW(gabp::pw_marginals(ctx->p, w->Pd, w->hv, w->msg[w->cur], w->c, nullptr, nullptr, 1, ctx->stream),
          "pairwise mean");
    CK_PW(gabp::launch_residual_mu(ctx->p, ctx->stream), "residual kernels");
    CK_PW(cudaMemcpyAsync(ctx->hscal, ctx->p.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "residual copy");
    CK_PW(cudaStreamSynchronize(ctx->stream), "residual sync");
    const double r2 = ctx->hscal[0], b2 = ctx->hscal[1];
    *rel = b2 > 0.0 ? std::sqrt(r2) / std::sqrt(b2) : std::sqrt(r2);
    return GABP_OK;
}

int gabp_pw_reset(gabp_pw *w) {
    if (!w) return GABP_ERR_ARG;
    DeviceGuard dg(w->ctx->dev);
    CK_PW(gabp::pw_zero(w->ctx->p, w->msg[0], w->ctx->stream), "pairwise reset");
    CK_PW(cudaStreamSynchronize(w->ctx->stream), "pairwise reset sync");
    w->cur = 0;
    w->iters = 0;
    w->c = 1.0;
    return GABP_OK;
}

int64_t gabp_pw_iterations(const gabp_pw *w) { return w ? w->iters : -1; }

int gabp_pw_message_change(gabp_pw *w, double *out) {
    if (!w || !out) return w ? pfail(w, GABP_ERR_ARG, "mean_abs_change must not be NULL") : GABP_ERR_ARG;
    if (w->iters < 1) return pfail(w, GABP_ERR_STATE, "no iteration since the last reset");
    gabp_ctx *ctx = w->ctx;
    DeviceGuard dg(ctx->dev);
    CK_PW(gabp::pw_change(ctx->p, w->msg[0], w->msg[1], ctx->p.part, gabp::RES_BLOCKS, ctx->p.scal + 3, ctx->stream),
          "pairwise message change");
    CK_PW(cudaMemcpyAsync(ctx->hscal + 3, ctx->p.scal + 3, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
          "copy change");
    CK_PW(cudaStreamSynchronize(ctx->stream), "pairwise change sync");
    const int64_t e = gabp::pw_edge_count(ctx->p.nx, ctx->p.ny);
    *out = e > 0 ? ctx->hscal[3] / (2.0 * (double)e) : 0.0;
    return GABP_OK;
}

int gabp_pw_iterate_early_stop_ref(gabp_pw *w, int max_iters, double c, double learning_rate, double tau,
                                   double reference, int64_t *stopped_at, double *reference_used) {
    if (!w) return GABP_ERR_ARG;
    if (!(tau > 0.0) || max_iters < 3) return pfail(w, GABP_ERR_ARG, "tau > 0 and max_iters >= 3 required");
    if (!std::isfinite(reference)) return pfail(w, GABP_ERR_ARG, "reference must be finite");
    if (stopped_at) *stopped_at = 0;
    int rc = gabp_pw_iterate(w, 2, c, learning_rate);
    if (rc) return rc;
    double ref = 0.0, d = 0.0;
    if ((rc = gabp_pw_message_change(w, &ref))) return rc;
    if (!std::isfinite(ref)) return pfail(w, GABP_ERR_DIVERGED, "message change is not finite");
    if (reference > 0.0) ref = reference;
    if (reference_used) *reference_used = ref;
    for (int64_t t = 2;;) {
        if (t >= max_iters) return pfail(w, GABP_ERR_TIMEOUT, "max_iters reached before the early-stopping rule held");
        if ((rc = gabp_pw_iterate(w, 1, c, learning_rate))) return rc;
        ++t;
        if ((rc = gabp_pw_message_change(w, &d))) return rc;
        if (!std::isfinite(d)) return pfail(w, GABP_ERR_DIVERGED, "message change is not finite");
        if (d < tau * ref) {
            if (stopped_at) *stopped_at = t;
            return GABP_OK;
        }
    }
}

int gabp_pw_iterate_early_stop(gabp_pw *w, int max_iters, double c, double learning_rate, double tau,
                               int64_t *stopped_at) {
    return gabp_pw_iterate_early_stop_ref(w, max_iters, c, learning_rate, tau, 0.0, stopped_at, nullptr);
}

int gabp_pw_upscale(gabp_pw *fine, const gabp_pw *coarse) {
    if (!fine || !coarse) return fine ? pfail(fine, GABP_ERR_ARG, "coarse must not be NULL") : GABP_ERR_ARG;
    gabp_pw *w = fine;   // error reporting (CK_PW)
    gabp_ctx *fc = fine->ctx, *cc = coarse->ctx;
    if (fc->p.prec != cc->p.prec || fc->dev != cc->dev)
        return pfail(fine, GABP_ERR_ARG, "levels of different precision or device");
    DeviceGuard dg(fc->dev);
    // the coarse level's messages are complete on its stream before the fine level reads them
    CK_PW(cudaStreamSynchronize(cc->stream), "coarse sync");
    CK_PW(gabp::pw_upscale(fc->p, cc->p, coarse->msg[coarse->cur], fine->msg[0], fc->stream), "pairwise upscale");
    CK_PW(cudaStreamSynchronize(fc->stream), "pairwise upscale sync");
    fine->cur = 0;
    fine->iters = 0;
    fine->c = coarse->c;   // the messages carry the coarse level's weight until the next iteration
    return GABP_OK;
}

const char *gabp_pw_last_error(const gabp_pw *w) { return w ? w->err.c_str() : ""; }

void gabp_pw_destroy(gabp_pw *w) {
    if (!w) return;
    DeviceGuard dg(w->ctx->dev);
    pw_free(w);
    delete w;
}

int gabp_wsnet_warm_start(gabp_ctx *c, gabp_wsnet *net) {
    NvtxRange nvtx_range("gabp_wsnet_warm_start");
    if (!c || !net) return c ? fail(c, GABP_ERR_ARG, "net must not be NULL") : GABP_ERR_ARG;
    if (gabp::wsnet_device(net) != c->dev) return fail(c, GABP_ERR_ARG, "network and context on different devices");
    if (c->p.order == 2) return fail(c, GABP_ERR_STATE, "warm starts are not available for the alpha = 4 prior");
    DeviceGuard g(c->dev);
    int rc = ws_ensure_input(c);
    if (rc) return rc;
    const int Hp = pad8(c->p.ny), Wp = pad8(c->p.nx);
    CK(gabp::launch_ws_input(c->p, c->yscale, c->kappa, Hp, Wp, c->ws_x, c->stream), "network input");
    float *out = nullptr;
    std::string err;
    rc = gabp::wsnet_forward_device(net, c->ws_x, 1, Hp, Wp, &out, c->stream, err);
    if (rc) return fail(c, rc, "network forward: " + err);
    const int64_t n = c->p.n;
    if (c->p.prec == 0) {   // FP32 messages: decode and initialise in FP32 (stage holds n float2)
        CK(gabp::launch_ws_init_f32(c->p, 0, c->yscale, Wp, out, (float2 *)c->stage, c->stream), "warm init kernels");
    } else {
        CK(gabp::launch_ws_decode(c->p, c->yscale, Wp, out, c->stage, c->stage + n, c->stream), "decode");
        CK(gabp::launch_init_warm(c->p, 0, c->stage, c->stage + n, c->stream), "warm init kernels");
    }
    CK(cudaStreamSynchronize(c->stream), "warm start sync");
    if (gabp::wsnet_take_device_error(net)) return fail(c, GABP_ERR_TIMEOUT, "network kernel wait ran out");
    c->cur = 0;
    c->iters = 0;
    c->last_res = NAN;
    return GABP_OK;
}

}  // extern "C"
