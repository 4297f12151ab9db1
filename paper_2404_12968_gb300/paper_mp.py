"""The paper's message passing as the paper runs it (Alg. 2, "Re-weighted message passing with
multigrid, damping, and early stopping"): the pairwise re-weighted form (App. A) with weight c
and learning rate eta, levels from a coarse base grid to the target grid (Sec. 3.2
"Multigrid"; every finer level starts from the coarser level's edge values, "Upscale
Messages"), and every level stopped by the early-stopping rule (App. B).

Levels: level k has spacing 2^k target cells, ceil(N / 2^k) nodes per axis, and the same SPDE
prior discretised there (kappa_k = 2^k kappa, gamma_k = gamma / 4^k).  An observation at a
grid point enters level k only if its location is a level-k grid point (the paper's rule;
grid-point observations only).  A level whose rule does not hold within max_iters iterations
(the paper's T) passes its messages on as they are.

Every step runs in the library's kernels; this module only builds the levels and sequences
the calls.
"""
from __future__ import annotations

import math

import numpy as np

from . import GabpError, GABP_ERR_TIMEOUT, Pairwise, Solver


def level_count(nx: int, ny: int, base: int = 32) -> int:
    """Levels from the target grid down to a base grid of about base x base nodes."""
    n = min(nx, ny)
    return max(1, int(math.floor(math.log2(n / base) + 1e-9)) + 1) if n > base else 1


def level_observations(obs_x, obs_y, y, noise_var, k: int):
    """The grid-point observations that coincide with level-k grid points, in level-k
    coordinates."""
    s = 1 << k
    ox = np.asarray(obs_x, np.float64)
    oy = np.asarray(obs_y, np.float64)
    if np.any(ox != np.round(ox)) or np.any(oy != np.round(oy)):
        raise ValueError("the paper's multigrid rule is for grid-point observations")
    sel = (np.mod(ox, s) == 0) & (np.mod(oy, s) == 0)
    return ox[sel] / s, oy[sel] / s, np.asarray(y, np.float64)[sel], np.asarray(noise_var, np.float64)[sel]


def solve(problem, *, c: float = 10.0, learning_rate: float = 0.6, tau: float = 1e-3, levels: int | None = None,
          base: int = 32, max_iters: int = 10000, precision: str = "fp32", gamma: float | None = None,
          device: int = 0, reference: str = "level"):
    """Run Alg. 2 on a problem with grid-point observations.  Returns (mean, variance, stops)
    with stops[k] the stopping iteration of level k (max_iters where the rule did not hold).

    ``reference`` reads which m_1, m_2 the early-stopping rule (App. B) compares against:
    "level" = the first two iterations of each level, "first" = those of the coarsest level,
    passed on to every finer level."""
    if reference not in ("level", "first"):
        raise ValueError(reference)
    nx, ny = int(problem.nx), int(problem.ny)
    g = float(gamma if gamma is not None else getattr(problem, "gamma", 1.0))
    L = levels if levels is not None else level_count(nx, ny, base)
    stops = {}
    first_ref = None
    prev = None   # (solver, pairwise) of the coarser level
    try:
        for k in range(L - 1, -1, -1):
            s = 1 << k
            nxk, nyk = -(-nx // s), -(-ny // s)
            ox, oy, yk, vk = level_observations(problem.obs_x, problem.obs_y, problem.y, problem.noise_var, k)
            sol = Solver(nx=nxk, ny=nyk, kappa=problem.kappa * s, obs_xy=np.stack([ox, oy], axis=1), y=yk,
                         noise_var=vk, gamma=g / (s * s), precision=precision, device=device)
            pw = Pairwise(sol)
            if prev is not None:
                pw.upscale_from(prev[1])
                prev[1].close()
                prev[0].close()
            try:
                stops[k] = pw.iterate_early_stop(max_iters, c, learning_rate, tau, first_ref)
            except GabpError as e:
                if e.code != GABP_ERR_TIMEOUT:
                    raise
                stops[k] = max_iters
            if reference == "first" and first_ref is None:
                first_ref = pw.reference_used
            prev = (sol, pw)
        mean, var = prev[1].marginals()
        return mean, var, stops
    finally:
        if prev is not None:
            prev[1].close()
            prev[0].close()
