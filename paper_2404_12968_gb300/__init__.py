"""GB300 Gaussian belief propagation for spatial data assimilation.

Python binding of the C ABI in ``include/gabp.h`` (libgabp.so).  The functions keep the C
names (``gabp_create``, ``gabp_iterate``, ``gabp_marginals``, ``gabp_residual``, ...) and
only marshal arguments; ``Solver`` is a small convenience wrapper that owns a context.

Array arguments may be NumPy arrays (host memory) or CUDA torch tensors (device memory);
both must be contiguous float64 where the C ABI takes ``double*``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (GABP_ERR_ARG, GABP_ERR_CUDA, GABP_ERR_DIVERGED, GABP_ERR_OOM,  # noqa: F401
                   GABP_ERR_STATE, GABP_ERR_TIMEOUT, GABP_FP32, GABP_FP64, GABP_INIT_COLD,
                   GABP_INIT_PAPER, GABP_KERNEL_AUTO, GABP_KERNEL_FUSED, GABP_KERNEL_SPLIT, GABP_KERNEL_TMA,
                   GABP_KERNEL_SWEEP,
                   GABP_OK, GabpError)

__all__ = [
    "gabp_default_options", "gabp_create", "gabp_iterate", "gabp_marginals", "gabp_residual",
    "gabp_warm_start", "gabp_reset", "gabp_set_prior_mean",
    "gabp_message_bytes", "gabp_get_messages",
    "gabp_set_messages", "gabp_get_stats", "gabp_destroy", "gabp_residual_noalloc",
    "gabp_batch_create", "gabp_batch_iterate", "gabp_batch_residuals", "gabp_batch_marginals",
    "gabp_batch_get_stats", "gabp_batch_strip_height", "gabp_batch_destroy",
    "gabp_wsnet_create", "gabp_wsnet_param_count", "gabp_wsnet_get_params", "gabp_wsnet_set_params",
    "gabp_wsnet_forward", "gabp_wsnet_gradients", "gabp_wsnet_train_step", "gabp_wsnet_destroy",
    "gabp_wsnet_set_kernels", "GABP_WSNET_TCGEN05", "GABP_WSNET_MMA_SYNC",
    "gabp_wsnet_input_shape", "gabp_wsnet_sample", "gabp_batch_input_shape", "gabp_batch_wsnet_sample",
    "gabp_wsnet_warm_start", "Solver", "Batch", "WarmStartNet", "GabpError",
    "gabp_mg_create", "gabp_mg_warm_start", "gabp_mg_destroy", "Multigrid",
    "gabp_message_change", "gabp_iterate_early_stop",
    "gabp_pw_create", "gabp_pw_iterate", "gabp_pw_marginals", "gabp_pw_residual", "gabp_pw_reset",
    "gabp_pw_destroy", "Pairwise",
]


def _ptr(a):
    """Address of a contiguous float64 host array or CUDA tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(rc: int, ctx=None, create: bool = False):
    if rc != GABP_OK:
        L = _lib.load()
        msg = (L.gabp_create_error() if create else L.gabp_last_error(ctx)) or b""
        raise GabpError(rc, msg.decode(errors="replace"))


def gabp_default_options(**over) -> _lib.gabp_options:
    o = _lib.gabp_options()
    _lib.load().gabp_default_options(ctypes.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def gabp_create(nx: int, ny: int, kappa: float, obs_xy, y, noise_var, *, gamma: float = 1.0, alpha: int = 2,
                h: float = 1.0, options: _lib.gabp_options | None = None, **opts) -> int:
    """Create a context; returns its handle.  ``obs_xy`` is (m, 2) float64 host data in grid
    units; ``alpha`` the SPDE exponent (2: cell factors = rows of L, 4: rows of L^2); ``h`` the
    grid spacing of the prior's Laplacian."""
    L = _lib.load()
    obs_xy = np.ascontiguousarray(obs_xy, np.float64).reshape(-1)
    y = np.ascontiguousarray(y, np.float64).reshape(-1)
    noise_var = np.ascontiguousarray(noise_var, np.float64).reshape(-1)
    m = y.shape[0]
    if obs_xy.shape[0] != 2 * m or noise_var.shape[0] != m:
        raise ValueError("obs_xy must be (m, 2) and noise_var (m,)")
    o = options if options is not None else gabp_default_options(**opts)
    prior = _lib.gabp_prior(gamma, 0, int(alpha))
    handle = ctypes.c_void_p()
    rc = L.gabp_create(ctypes.byref(handle), _lib.gabp_grid(nx, ny, float(h)), float(kappa), ctypes.byref(prior),
                       m, obs_xy.ctypes.data if m else None, y.ctypes.data if m else None,
                       noise_var.ctypes.data if m else None, ctypes.byref(o))
    _check(rc, create=True)
    return handle.value


def gabp_iterate(ctx: int, n_iters: int, damping: float) -> None:
    _check(_lib.load().gabp_iterate(ctx, int(n_iters), float(damping)), ctx)


def gabp_marginals(ctx: int, mean, var=None) -> None:
    _check(_lib.load().gabp_marginals(ctx, _ptr(mean), _ptr(var)), ctx)


def gabp_residual(ctx: int) -> float:
    out = ctypes.c_double()
    _check(_lib.load().gabp_residual(ctx, ctypes.byref(out)), ctx)
    return out.value


def gabp_warm_start(ctx: int, mu0, lam0) -> None:
    _check(_lib.load().gabp_warm_start(ctx, _ptr(mu0), _ptr(lam0)), ctx)


def gabp_reset(ctx: int) -> None:
    _check(_lib.load().gabp_reset(ctx), ctx)


def gabp_set_prior_mean(ctx: int, f_b) -> None:
    """Prior mean f_b (nx*ny float64, host array or CUDA tensor; None = zero)."""
    _check(_lib.load().gabp_set_prior_mean(ctx, _ptr(f_b)), ctx)


def gabp_message_bytes(ctx: int) -> int:
    return int(_lib.load().gabp_message_bytes(ctx))


def gabp_get_messages(ctx: int, buf) -> None:
    _check(_lib.load().gabp_get_messages(ctx, _ptr(buf)), ctx)


def gabp_set_messages(ctx: int, buf) -> None:
    _check(_lib.load().gabp_set_messages(ctx, _ptr(buf)), ctx)


def gabp_get_stats(ctx: int) -> dict:
    s = _lib.gabp_stats()
    _check(_lib.load().gabp_get_stats(ctx, ctypes.byref(s)), ctx)
    return {f: getattr(s, f) for f, _ in s._fields_}


def gabp_destroy(ctx: int) -> None:
    if ctx:
        _lib.load().gabp_destroy(ctx)


def _device_f64_count(t, name: str) -> int:
    """Number of elements of ``t``, which must be a contiguous float64 CUDA tensor on the current
    device (the allocation-free entry point reads it from the GPU as it is)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must live on the current CUDA device")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 tensor")
    return int(t.numel())


def gabp_residual_noalloc(nx: int, ny: int, kappa: float, obs_xy, y, noise_var, mean, *,
                          gamma: float = 1.0, stream=None) -> float:
    """Relative residual of ``mean`` without any allocation by the library.

    ``obs_xy`` (2m), ``y``, ``noise_var`` (m) and ``mean`` (nx*ny) are contiguous float64 CUDA
    tensors on the current device; the observations must be sorted by base cell.  ``stream`` is
    a ``cudaStream_t`` value (e.g. ``torch.cuda.current_stream().cuda_stream``) or None."""
    L = _lib.load()
    m = _device_f64_count(y, "y")
    if _device_f64_count(mean, "mean") != nx * ny:
        raise ValueError(f"mean must hold nx * ny = {nx * ny} values")
    if _device_f64_count(obs_xy, "obs_xy") != 2 * m or _device_f64_count(noise_var, "noise_var") != m:
        raise ValueError("obs_xy must hold 2 m values and noise_var m values (m = len(y))")
    out = ctypes.c_double()
    rc = L.gabp_residual_noalloc(_lib.gabp_grid(nx, ny, 1.0), float(kappa), float(gamma), m,
                                 _ptr(obs_xy) if m else None, _ptr(y) if m else None,
                                 _ptr(noise_var) if m else None, _ptr(mean), ctypes.byref(out), stream)
    if rc != GABP_OK:
        raise GabpError(rc, (L.gabp_residual_noalloc_error() or b"").decode(errors="replace"))
    return out.value


def _bcheck(rc: int, b):
    if rc != GABP_OK:
        raise GabpError(rc, (_lib.load().gabp_batch_last_error(b) or b"").decode(errors="replace"))


def gabp_batch_create(problems, **opts) -> int:
    """Create a batch from ``gabp_synth.Problem``-like objects; returns its handle."""
    L = _lib.load()
    keep = []
    arr = (_lib.gabp_problem * len(problems))()
    for i, pr in enumerate(problems):
        xy = np.ascontiguousarray(np.stack([pr.obs_x, pr.obs_y], axis=1).reshape(-1), np.float64)
        y = np.ascontiguousarray(pr.y, np.float64)
        nv = np.ascontiguousarray(pr.noise_var, np.float64)
        keep += [xy, y, nv]
        m = y.shape[0]
        arr[i] = _lib.gabp_problem(_lib.gabp_grid(pr.nx, pr.ny, 1.0), float(pr.kappa),
                                   float(getattr(pr, "gamma", 1.0)), m, xy.ctypes.data if m else None,
                                   y.ctypes.data if m else None, nv.ctypes.data if m else None)
    o = gabp_default_options(**opts)
    h = ctypes.c_void_p()
    rc = L.gabp_batch_create(ctypes.byref(h), len(problems), arr, ctypes.byref(o))
    if rc != GABP_OK:
        raise GabpError(rc, (L.gabp_batch_last_error(None) or b"").decode(errors="replace"))
    return h.value


def gabp_batch_iterate(b: int, n_iters: int, damping: float) -> None:
    _bcheck(_lib.load().gabp_batch_iterate(b, int(n_iters), float(damping)), b)


def gabp_batch_residuals(b: int, count: int) -> np.ndarray:
    out = np.empty(count)
    _bcheck(_lib.load().gabp_batch_residuals(b, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), b)
    return out


def gabp_batch_marginals(b: int, index: int, mean, var=None) -> None:
    _bcheck(_lib.load().gabp_batch_marginals(b, int(index), _ptr(mean), _ptr(var)), b)


def gabp_batch_get_stats(b: int, index: int) -> dict:
    s = _lib.gabp_stats()
    _bcheck(_lib.load().gabp_batch_get_stats(b, int(index), ctypes.byref(s)), b)
    return {f: getattr(s, f) for f, _ in s._fields_}


def gabp_batch_strip_height(b: int) -> int:
    return int(_lib.load().gabp_batch_strip_height(b))


def gabp_batch_destroy(b: int) -> None:
    if b:
        _lib.load().gabp_batch_destroy(b)


class Batch:
    """Owns a batch of independent problems iterated together (one persistent launch per
    iteration)."""

    def __init__(self, problems, **opts):
        self.sizes = [(int(p.nx), int(p.ny)) for p in problems]
        self.handle = gabp_batch_create(problems, **opts)

    def __len__(self):
        return len(self.sizes)

    def iterate(self, n_iters: int, damping: float) -> "Batch":
        gabp_batch_iterate(self.handle, n_iters, damping)
        return self

    def residuals(self) -> np.ndarray:
        return gabp_batch_residuals(self.handle, len(self))

    def marginals(self, index: int, want_var: bool = False):
        nx, ny = self.sizes[index]
        mean = np.empty(nx * ny)
        var = np.empty(nx * ny) if want_var else None
        gabp_batch_marginals(self.handle, index, mean, var)
        return mean, var

    def stats(self, index: int) -> dict:
        return gabp_batch_get_stats(self.handle, index)

    @property
    def strip_height(self) -> int:
        """Tile height of the TMA kernel (14, 22, 30) or strip height of the sweep kernel."""
        return gabp_batch_strip_height(self.handle)

    @property
    def kernel(self) -> int:
        """GABP_KERNEL_TMA or GABP_KERNEL_SWEEP: the kernel iterating this batch."""
        return self.stats(0)["kernel"]

    @property
    def kernel_name(self) -> str:
        return "k_fused_tma (batched)" if self.kernel == GABP_KERNEL_TMA else "k_sweep_batch"

    def close(self):
        if getattr(self, "handle", None):
            gabp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def gabp_message_change(ctx: int) -> float:
    """Mean |m_t - m_{t-1}| over both components of every edge (the early-stopping quantity)."""
    d = ctypes.c_double()
    _check(_lib.load().gabp_message_change(ctx, ctypes.byref(d)), ctx)
    return d.value


def gabp_iterate_early_stop(ctx: int, max_iters: int, damping: float, tau: float = 1e-3,
                            check_every: int = 1) -> int:
    """Iterate under the paper's early-stopping rule (App. B); returns the stopping iteration."""
    t = ctypes.c_int64()
    _check(_lib.load().gabp_iterate_early_stop(ctx, max_iters, damping, tau, check_every, ctypes.byref(t)), ctx)
    return t.value


def _pcheck(rc: int, pw):
    if rc != GABP_OK:
        raise GabpError(rc, (_lib.load().gabp_pw_last_error(pw) or b"").decode(errors="replace"))


def gabp_pw_create(ctx: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.load().gabp_pw_create(ctypes.byref(h), ctx), ctx)
    return h.value


def gabp_pw_iterate(pw: int, n_iters: int, c: float = 10.0, learning_rate: float = 0.6) -> None:
    _pcheck(_lib.load().gabp_pw_iterate(pw, n_iters, c, learning_rate), pw)


def gabp_pw_marginals(pw: int, mean, var=None) -> None:
    _pcheck(_lib.load().gabp_pw_marginals(pw, _ptr(mean), _ptr(var) if var is not None else None), pw)


def gabp_pw_residual(pw: int) -> float:
    r = ctypes.c_double()
    _pcheck(_lib.load().gabp_pw_residual(pw, ctypes.byref(r)), pw)
    return r.value


def gabp_pw_reset(pw: int) -> None:
    _pcheck(_lib.load().gabp_pw_reset(pw), pw)


def gabp_pw_destroy(pw: int) -> None:
    if pw:
        _lib.load().gabp_pw_destroy(pw)


class Pairwise:
    """The paper's pairwise re-weighted message passing (App. A) on a Solver's problem.
    The Solver must outlive it."""

    def __init__(self, solver: "Solver"):
        self.n = solver.nx * solver.ny
        self.handle = gabp_pw_create(solver.ctx)

    def iterate(self, n_iters: int, c: float = 10.0, learning_rate: float = 0.6) -> None:
        gabp_pw_iterate(self.handle, n_iters, c, learning_rate)

    def marginals(self, want_var: bool = True):
        mean = np.empty(self.n, np.float64)
        var = np.empty(self.n, np.float64) if want_var else None
        gabp_pw_marginals(self.handle, mean, var)
        return mean, var

    def message_change(self) -> float:
        """mean |m_t - m_{t-1}| over every pair-factor message (the early-stopping quantity)."""
        d = ctypes.c_double()
        _pcheck(_lib.load().gabp_pw_message_change(self.handle, ctypes.byref(d)), self.handle)
        return d.value

    def iterate_early_stop(self, max_iters: int, c: float = 10.0, learning_rate: float = 0.6,
                           tau: float = 1e-3, reference: float | None = None) -> int:
        """Iterate under the early-stopping rule (App. B); returns the stopping iteration.
        ``reference`` (> 0) replaces this call's own change between its iterations 1 and 2;
        the reference the rule used is left in ``self.reference_used``."""
        t = ctypes.c_int64()
        used = ctypes.c_double()
        used.value = float("nan")
        rc = _lib.load().gabp_pw_iterate_early_stop_ref(self.handle, int(max_iters), float(c), float(learning_rate),
                                                        float(tau), float(reference or 0.0), ctypes.byref(t),
                                                        ctypes.byref(used))
        self.reference_used = used.value     # set once iterations 1 and 2 ran, also on a timeout
        _pcheck(rc, self.handle)
        return t.value

    def upscale_from(self, coarse: "Pairwise") -> None:
        """Initialise this level's messages from the coarser level's ("Upscale Messages")."""
        _pcheck(_lib.load().gabp_pw_upscale(self.handle, coarse.handle), self.handle)

    def residual(self) -> float:
        return gabp_pw_residual(self.handle)

    def reset(self) -> None:
        gabp_pw_reset(self.handle)

    @property
    def iterations(self) -> int:
        return int(_lib.load().gabp_pw_iterations(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            gabp_pw_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gabp_mg_create(ctx: int, levels: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.load().gabp_mg_create(ctypes.byref(h), ctx, levels), ctx)
    return h.value


def gabp_mg_warm_start(mg: int, damping: float, tol: float, max_iters: int) -> dict:
    """Run the coarse levels and warm-start the target context; per-level statistics."""
    st = _lib.gabp_mg_stats()
    rc = _lib.load().gabp_mg_warm_start(mg, damping, tol, max_iters, ctypes.byref(st))
    if rc != GABP_OK:
        raise GabpError(rc, (_lib.load().gabp_mg_last_error(mg) or b"").decode(errors="replace"))
    L = st.levels
    return {"levels": L, "iterations": [int(st.iterations[k]) for k in range(L)],
            "damping": [float(st.damping[k]) for k in range(L)], "residual": [float(st.residual[k]) for k in range(L)],
            "converged": [bool(st.converged[k]) for k in range(L)]}


def gabp_mg_destroy(mg: int) -> None:
    if mg:
        _lib.load().gabp_mg_destroy(mg)


class Multigrid:
    """Coarse levels of a Solver's problem for the multigrid warm start (Sec. 3.2, Alg. 2).
    The Solver must outlive it.  Entry k of the per-level lists is level k (0 unused)."""

    def __init__(self, solver: "Solver", levels: int):
        self.handle = gabp_mg_create(solver.ctx, levels)

    def warm_start(self, damping: float = 0.3, tol: float = 1e-5, max_iters: int = 100000) -> dict:
        return gabp_mg_warm_start(self.handle, damping, tol, max_iters)

    def close(self):
        if getattr(self, "handle", None):
            gabp_mg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _wcheck(rc: int, net):
    if rc != GABP_OK:
        L = _lib.load()
        msg = L.gabp_wsnet_last_error(net) if net else L.gabp_wsnet_create_error()
        raise GabpError(rc, (msg or b"").decode(errors="replace"))


def gabp_wsnet_create(seed: int = 0, device: int = -1) -> int:
    h = ctypes.c_void_p()
    _wcheck(_lib.load().gabp_wsnet_create(ctypes.byref(h), int(seed), int(device)), None)
    return h.value


def gabp_wsnet_param_count(net: int) -> int:
    return int(_lib.load().gabp_wsnet_param_count(net))


def gabp_wsnet_get_params(net: int, out) -> None:
    _wcheck(_lib.load().gabp_wsnet_get_params(net, _ptr(out)), net)


def gabp_wsnet_set_params(net: int, params) -> None:
    _wcheck(_lib.load().gabp_wsnet_set_params(net, _ptr(params)), net)


GABP_WSNET_TCGEN05 = 0
GABP_WSNET_MMA_SYNC = 1


def gabp_wsnet_set_kernels(net: int, kernels: int) -> None:
    _wcheck(_lib.load().gabp_wsnet_set_kernels(net, kernels), net)


def gabp_wsnet_forward(net: int, x, B: int, H: int, W: int, out) -> None:
    _wcheck(_lib.load().gabp_wsnet_forward(net, _ptr(x), B, H, W, _ptr(out)), net)


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = _ptr(t)
    return arr


def gabp_wsnet_gradients(net: int, xs, ts, H: int, W: int, grads=None) -> float:
    loss = ctypes.c_float()
    _wcheck(_lib.load().gabp_wsnet_gradients(net, _ptr_array(xs), _ptr_array(ts), len(xs), H, W, _ptr(grads),
                                             ctypes.byref(loss)), net)
    return loss.value


def gabp_wsnet_train_step(net: int, xs, ts, H: int, W: int, lr: float) -> float:
    loss = ctypes.c_float()
    _wcheck(_lib.load().gabp_wsnet_train_step(net, _ptr_array(xs), _ptr_array(ts), len(xs), H, W, float(lr),
                                              ctypes.byref(loss)), net)
    return loss.value


def gabp_wsnet_destroy(net: int) -> None:
    if net:
        _lib.load().gabp_wsnet_destroy(net)


def gabp_wsnet_input_shape(ctx: int):
    H, W, sc = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(_lib.load().gabp_wsnet_input_shape(ctx, ctypes.byref(H), ctypes.byref(W), ctypes.byref(sc)), ctx)
    return H.value, W.value, sc.value


def gabp_wsnet_sample(ctx: int, x_out=None, t_out=None) -> None:
    _check(_lib.load().gabp_wsnet_sample(ctx, _ptr(x_out), _ptr(t_out)), ctx)


def gabp_batch_input_shape(b: int, index: int):
    H, W, sc = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _bcheck(_lib.load().gabp_batch_input_shape(b, int(index), ctypes.byref(H), ctypes.byref(W), ctypes.byref(sc)), b)
    return H.value, W.value, sc.value


def gabp_batch_wsnet_sample(b: int, index: int, x_out=None, t_out=None) -> None:
    _bcheck(_lib.load().gabp_batch_wsnet_sample(b, int(index), _ptr(x_out), _ptr(t_out)), b)


def gabp_wsnet_warm_start(ctx: int, net: int) -> None:
    _check(_lib.load().gabp_wsnet_warm_start(ctx, net), ctx)


class WarmStartNet:
    """Owns a warm-start network (weights on the GPU)."""

    def __init__(self, seed: int = 0, device: int = -1):
        self.handle = gabp_wsnet_create(seed, device)
        self.nparam = gabp_wsnet_param_count(self.handle)

    def params(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        gabp_wsnet_get_params(self.handle, out)
        return out

    def set_params(self, params) -> None:
        gabp_wsnet_set_params(self.handle, np.ascontiguousarray(params, np.float32))

    def save(self, path: str) -> None:
        np.save(path, self.params())

    def load(self, path: str) -> None:
        self.set_params(np.load(path))

    def close(self):
        if getattr(self, "handle", None):
            gabp_wsnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owns one context.  ``Solver(problem, precision='fp32')`` with a ``gabp_synth.Problem``-like
    object (fields nx, ny, kappa, obs_x, obs_y, y, noise_var)."""

    def __init__(self, problem=None, *, nx=None, ny=None, kappa=None, obs_xy=None, y=None,
                 noise_var=None, precision: str = "fp32", gamma: float = 1.0, alpha: int = 2, h: float = 1.0,
                 **opts):
        if problem is not None:
            nx, ny, kappa = problem.nx, problem.ny, problem.kappa
            obs_xy = np.stack([problem.obs_x, problem.obs_y], axis=1)
            y, noise_var = problem.y, problem.noise_var
        opts.setdefault("precision", GABP_FP64 if precision == "fp64" else GABP_FP32)
        self.nx, self.ny = int(nx), int(ny)
        self.ctx = gabp_create(self.nx, self.ny, kappa, obs_xy, y, noise_var, gamma=gamma, alpha=alpha, h=h, **opts)

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def iterate(self, n_iters: int, damping: float) -> "Solver":
        gabp_iterate(self.ctx, n_iters, damping)
        return self

    def residual(self) -> float:
        return gabp_residual(self.ctx)

    def marginals(self, out_mean=None, out_var=None, want_var: bool = True):
        mean = out_mean if out_mean is not None else np.empty(self.n)
        var = out_var if out_var is not None else (np.empty(self.n) if want_var else None)
        gabp_marginals(self.ctx, mean, var)
        return mean, var

    def learned_warm_start(self, net: "WarmStartNet") -> None:
        gabp_wsnet_warm_start(self.ctx, net.handle)

    def warm_start(self, mu0, lam0) -> None:
        gabp_warm_start(self.ctx, np.ascontiguousarray(mu0, np.float64).reshape(-1)
                        if isinstance(mu0, np.ndarray) else mu0,
                        np.ascontiguousarray(lam0, np.float64).reshape(-1)
                        if isinstance(lam0, np.ndarray) else lam0)

    def reset(self) -> None:
        gabp_reset(self.ctx)

    def set_prior_mean(self, f_b) -> None:
        gabp_set_prior_mean(self.ctx, np.ascontiguousarray(f_b, np.float64).reshape(-1)
                            if isinstance(f_b, np.ndarray) else f_b)

    def message_change(self) -> float:
        return gabp_message_change(self.ctx)

    def iterate_early_stop(self, max_iters: int, damping: float, tau: float = 1e-3, check_every: int = 1) -> int:
        return gabp_iterate_early_stop(self.ctx, max_iters, damping, tau, check_every)

    def get_messages(self) -> np.ndarray:
        buf = np.empty(gabp_message_bytes(self.ctx), np.uint8)
        gabp_get_messages(self.ctx, buf)
        return buf

    def set_messages(self, buf: np.ndarray) -> None:
        gabp_set_messages(self.ctx, np.ascontiguousarray(buf))

    def stats(self) -> dict:
        return gabp_get_stats(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            gabp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
