"""Multigrid warm start of GaBP (TEST INFRASTRUCTURE ONLY).

Sec. 3.2 "Multigrid" and Alg. 2 ("Multigrid MP", "Upscale Messages"): solve the problem on a
coarse grid first, then repeatedly double the grid, starting each finer level from the
previous level's converged state, until the target grid is reached.

Readings (the paper states the procedure for grid-point observations and a generic grid):

* Level k (k = 0 is the target grid) has spacing 2^k target cells and ceil(N / 2^k) nodes
  per axis; node (i, j) of level k sits at target coordinates (2^k i, 2^k j).  The prior is
  the same SPDE discretised at that spacing: with the unit-spacing stencil of the target
  level this is kappa_k = 2^k kappa and gamma_k = gamma / 4^k (the discrete white noise of a
  cell of area h^2 has precision gamma h^2, and L_h = (kappa^2 - Delta_h) = h^-2 L_1 at
  kappa h).
* Observations carry continuous locations here, so the paper's "introduced at a level where
  the location coincides with a grid point" would leave the coarse levels without data.
  Every observation is introduced at every level instead, at its location in that level's
  coordinates (x / 2^k, y / 2^k, clamped to the level's last node), with its own value and
  noise variance.
* A level whose GaBP diverges cannot deliver the converged state the procedure passes on.
  Dense observations on a very coarse grid do make GaBP diverge at the damping that suits
  the target level.  A level whose final relative residual is not finite or not below 1
  (worse than mu = 0) is re-run from its starting state with the damping (1 + beta) / 2, up
  to three times; if it still fails, the next level starts from this level's own starting
  state (cold when there is none).
* "Upscale Messages" initialises the finer level so that its marginals equal the coarser
  level's (the paper states that copying the edge values is equivalent to this): every node
  of level k - 1 takes the marginal (mean, precision) of its parent node
  (floor(i / 2), floor(j / 2)) of level k, and its messages are set by the warm-start rule
  (precision lambda0 / (number of factor slots at the node), information mu0 * that).
"""
from __future__ import annotations

import numpy as np

from . import build_factors, gabp, residual


def level_shape(nx: int, ny: int, k: int):
    """Nodes per axis of level k: ceil(N / 2^k)."""
    s = 1 << k
    return -(-nx // s), -(-ny // s)


def level_problem(nx, ny, kappa, gamma, ox, oy, k: int):
    """(nx_k, ny_k, kappa_k, gamma_k, ox_k, oy_k) of level k."""
    s = 1 << k
    nxk, nyk = level_shape(nx, ny, k)
    oxk = np.minimum(np.asarray(ox, np.float64) / s, nxk - 1)
    oyk = np.minimum(np.asarray(oy, np.float64) / s, nyk - 1)
    return nxk, nyk, kappa * s, gamma / (s * s), oxk, oyk


def upscale(mu_c, var_c, nxc: int, nyc: int, nxf: int, nyf: int):
    """Marginals of the finer level from its parents: node (i, j) <- (floor(i/2), floor(j/2))."""
    mu_c = np.asarray(mu_c, np.float64).reshape(nyc, nxc)
    lam_c = 1.0 / np.asarray(var_c, np.float64).reshape(nyc, nxc)
    i = np.minimum(np.arange(nyf) // 2, nyc - 1)
    j = np.minimum(np.arange(nxf) // 2, nxc - 1)
    return mu_c[np.ix_(i, j)].reshape(-1), lam_c[np.ix_(i, j)].reshape(-1)


def solve_level(fl, beta: float, iters: int, mu0=None, lam0=None, retries: int = 3):
    """GaBP on one level from cold (mu0 None) or from marginals (mu0, lam0); a run that ends
    with a relative residual not finite or not below 1 is repeated with damping (1 + beta) / 2.
    Returns (mean, var, residual, damping used, converged)."""
    b = float(beta)
    for _ in range(retries + 1):
        if mu0 is None:
            m, v, _ = gabp(fl, b, iters, init="cold")
        else:
            m, v, _ = gabp(fl, b, iters, init="warm", mu0=mu0, lam0=lam0)
        r = residual(fl, m)
        if np.isfinite(r) and r < 1.0:
            return m, v, r, b, True
        b = 0.5 * (1.0 + b)
    return m, v, r, b, False


def multigrid_init(nx, ny, kappa, gamma, ox, oy, y, noise_var, levels: int, beta: float, iters):
    """Initial marginals (mu0, lam0) of the target level after levels - 1 coarse solves.

    ``iters``: GaBP iterations per coarse level (an int, or a dict level -> count), cold start
    on the coarsest level.  Also returns, per coarse level, (final relative residual, damping
    used, converged).
    """
    if levels < 2:
        raise ValueError("multigrid needs at least 2 levels")
    mu = lam = None
    info = {}
    for k in range(levels - 1, 0, -1):
        nxk, nyk, kk, gk, oxk, oyk = level_problem(nx, ny, kappa, gamma, ox, oy, k)
        fl = build_factors(nxk, nyk, kk, oxk, oyk, y, noise_var, gamma=gk)
        n_it = iters[k] if isinstance(iters, dict) else int(iters)
        m, v, r, b, ok = solve_level(fl, beta, n_it, mu, lam)
        info[k] = (r, b, ok)
        nxf, nyf = level_shape(nx, ny, k - 1)
        if ok:
            mu, lam = upscale(m, v, nxk, nyk, nxf, nyf)
        elif mu is not None:   # pass this level's own start on
            mu, lam = upscale(mu, 1.0 / lam, nxk, nyk, nxf, nyf)
    return mu, lam, info
