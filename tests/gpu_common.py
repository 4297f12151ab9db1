"""Helpers shared by the GPU tests: building the library on the GPU machine, running the CUDA path
and the oracle on the same seeded inputs, and decoding the message buffer."""
from __future__ import annotations

import os

import numpy as np

import gabp_synth


def ensure_built():
    from paper_2404_12968_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2404_12968_gb300.build import build
        build()
    _lib.load()


def rel_l2(a, b) -> float:
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_factors(orc, p: gabp_synth.Problem, gamma: float = 1.0):
    return orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, gamma)


def solver(p: gabp_synth.Problem, precision="fp32", **opts):
    from paper_2404_12968_gb300 import Solver
    return Solver(p, precision=precision, **opts)


def decode_messages(buf: np.ndarray, p: gabp_synth.Problem, precision="fp32"):
    """Split the opaque message buffer into prior planes (5, n, 2) and obs messages (m, 4, 2).

    The layout is the library's (documented in its device header): 5 prior planes of
    (eta, Lambda) pairs in outgoing order C, W, E, S, N, then per observation (in
    base-cell-sorted order) the (eta, Lambda) pairs of its four corners."""
    dt = np.float64 if precision == "fp64" else np.float32
    a = buf.view(dt)
    n, m = p.n, p.m
    prior = a[: 10 * n].reshape(5, n, 2)
    obs = a[10 * n: 10 * n + 8 * m].reshape(m, 4, 2)   # corner, (eta, Lambda)
    return prior, obs


def sorted_obs_order(orc, p: gabp_synth.Problem):
    """Stable order of observations by base cell (the oracle's own bilinear rule)."""
    i0, j0, w = orc.bilinear_base_weights(p.nx, p.ny, p.obs_x, p.obs_y)
    base = i0 * p.nx + j0
    return np.argsort(base, kind="stable"), base, w


def golden_writer():
    """``tests/golden/make_exact_means.py``, the script that wrote the stored exact means (the
    oracle alone), loaded as a module for its reader and its list of stored batch instances."""
    import importlib.util
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_exact_means.py")
    spec = importlib.util.spec_from_file_location("make_exact_means", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def load_exact_sample(name: str) -> dict:
    """A stored exact posterior mean at sampled nodes (``tests/golden/exact_mean_<name>.txt``)."""
    return golden_writer().load(name)


def same_inputs_as_sample(p: gabp_synth.Problem, g: dict) -> bool:
    """The problem the generator made here is the one the stored sample was solved for."""
    sums = {"sum_obs_x": p.obs_x, "sum_obs_y": p.obs_y, "sum_y": p.y, "sum_noise_var": p.noise_var}
    ok = p.nx == g["nx"] and p.ny == g["ny"] and p.m == g["m"] and abs(p.kappa - g["kappa"]) == 0.0
    for k, v in sums.items():
        ok = ok and abs(float(np.sum(v)) - g[k]) <= 1e-12 * max(1.0, abs(g[k]))
    return bool(ok)


def iterate_to_floor(step, residual, chunk: int, max_iters: int):
    """Iterate in chunks until the FP64 relative residual stops halving from one chunk to the
    next (the rounding floor of the message precision) or ``max_iters`` pass; returns the last
    residual and the iteration count."""
    best = np.inf
    its = 0
    res = np.inf
    while its < max_iters:
        step(chunk)
        its += chunk
        res = residual()
        if not res < 0.5 * best:
            break
        best = res
    return res, its


def iterate_until_settled(step, means, chunk: int, max_iters: int, tol: float = 1e-7):
    """Iterate in chunks until the means (an array, or a list of arrays: each must settle) change
    by less than tol (relative L2) from one chunk to the next, or max_iters pass; returns the
    iterations.  With FP32 messages the FP64 residual levels off near 5e-8 while the poorly
    observed smooth modes of a small-kappa problem are still converging, so it cannot tell when
    to stop."""
    def snap():
        m = means()
        return [np.array(x, copy=True) for x in (m if isinstance(m, list) else [m])]

    prev = snap()
    its = 0
    while its < max_iters:
        step(chunk)
        its += chunk
        cur = snap()
        change = max(float(np.linalg.norm(c - q) / max(np.linalg.norm(c), 1e-300)) for c, q in zip(cur, prev))
        prev = cur
        if change < tol:
            break
    return its
