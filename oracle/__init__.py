"""CPU FP64 oracle for the GaBP data-assimilation path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It is independent of the CUDA
library (no shared code, headers or constants) and never imports it.

Contents
--------
* ``build_factors``: the factor graph of the posterior as a generic list of rank-1
  factors ``exp(-(s/2)(a . x - r)^2)`` (with a prior mean f_b the cell factors' targets are
  r = a . f_b, ``with_prior_mean``):
    - prior (Sec. 3.1, P = gamma L^T L with L the finite-difference operator of App. C,
      Eq. for the discretised operator, extended to 2-D): one factor per cell i with
      a = row i of L, s = gamma, r = 0.  Zero-Neumann boundary, read as a cell-centred
      ghost equal to the boundary value, so row i of L has kappa^2 + deg(i) on the
      diagonal and -1 on each existing 4-neighbour (deg(i) = number of neighbours);
      alpha = 4 (Sec. 3.1, the SPDE with alpha/2 = 2; App. C, higher powers of the operator
      as powers of its matrix): the operator matrix is L^2, one factor per cell with
      a = row i of L^2 (13-point stencil), P = gamma (L^2)^T L^2;
    - observations (Sec. 3.2, "Including Observations", generalised to a row of H):
      one factor per observation with the four bilinear weights of its location,
      s = 1 / noise variance, r = y.
* ``gabp``: the synchronous damped serial GaBP of ``gabp_oracle.c``.
* ``exact_mean``: the exact posterior mean A^-1 b (banded Cholesky in C, or a sparse LU
  from scipy as a library step for larger grids); ``exact_variances``: diag(A^-1) by a
  dense inverse on small grids.
* ``residual``: ||b - A mu|| / ||b|| in FP64.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import build_oracle, library_path

__all__ = [
    "FactorList", "build_factors", "prior_factors", "with_prior_mean", "obs_factors", "bilinear_base_weights",
    "concat", "gabp", "init_messages", "factor_update", "beliefs", "apply_A", "rhs",
    "residual", "exact_mean", "exact_variances", "dense_A", "band_solve", "half_bandwidth", "lib",
]

_LIB = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load (building on first use) the oracle's C library."""
    global _LIB
    if _LIB is None:
        path = library_path()
        src = os.path.join(os.path.dirname(__file__), "gabp_oracle.c")
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
            build_oracle()
        L = ctypes.CDLL(path)
        L.orc_factor_update.argtypes = [ctypes.c_int, _f64p, ctypes.c_double, ctypes.c_double,
                                        _f64p, _f64p, _f64p, _f64p]
        L.orc_factor_update.restype = None
        L.orc_beliefs.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p,
                                  _f64p, _f64p]
        L.orc_beliefs.restype = None
        L.orc_init_messages.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _i64p, _i64p,
                                        _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_init_messages.restype = ctypes.c_int
        L.orc_gabp_run.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p,
                                   _f64p, ctypes.c_double, ctypes.c_int, _f64p, _f64p, _f64p, _f64p]
        L.orc_gabp_run.restype = ctypes.c_int
        L.orc_apply_A.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p,
                                  _f64p, _f64p]
        L.orc_apply_A.restype = None
        L.orc_rhs.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p, _f64p,
                              _f64p]
        L.orc_rhs.restype = None
        L.orc_band_solve.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p,
                                     ctypes.c_int64, _f64p]
        L.orc_band_solve.restype = ctypes.c_int
        L.orc_iterate_factors.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p, _f64p,
                                          ctypes.c_double, ctypes.c_int64, _i64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_iterate_factors.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


@dataclass
class FactorList:
    """Rank-1 factors in CSR form: factor f has slots ptr[f]..ptr[f+1]-1, each slot a
    (variable index, coefficient) pair; s[f] > 0 is the factor precision and r[f] its target."""
    n: int
    ptr: np.ndarray    # (nf+1,) int64
    var: np.ndarray    # (ne,) int64
    coef: np.ndarray   # (ne,) float64
    s: np.ndarray      # (nf,) float64
    r: np.ndarray      # (nf,) float64

    @property
    def nf(self) -> int:
        return int(self.s.shape[0])

    @property
    def ne(self) -> int:
        return int(self.var.shape[0])

    def check(self):
        assert self.ptr.dtype == np.int64 and self.var.dtype == np.int64
        assert self.ptr[0] == 0 and self.ptr[-1] == self.ne
        assert np.all(np.diff(self.ptr) >= 0)
        assert np.all((self.var >= 0) & (self.var < self.n))
        assert np.all(self.s > 0)
        return self


def concat(*lists: FactorList) -> FactorList:
    n = lists[0].n
    assert all(fl.n == n for fl in lists)
    ptrs, off = [np.zeros(1, np.int64)], 0
    for fl in lists:
        ptrs.append(fl.ptr[1:] + off)
        off += fl.ne
    return FactorList(n, np.concatenate(ptrs), np.concatenate([fl.var for fl in lists]),
                      np.concatenate([fl.coef for fl in lists]),
                      np.concatenate([fl.s for fl in lists]), np.concatenate([fl.r for fl in lists]))


# slot offsets (dx, dy) of the alpha = 4 cell factor: the cell, its 4 neighbours, the 4
# diagonal neighbours, the 4 nodes two steps away
_L2_OFFSETS = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1),
               (-2, 0), (2, 0), (0, -2), (0, 2)]


def prior_factors(nx: int, ny: int, kappa: float, gamma: float = 1.0, alpha: int = 2, h: float = 1.0) -> FactorList:
    """One factor per cell: a = row of L = kappa^2 I - Delta_h (zero-Neumann), or for alpha = 4
    a row of L^2.  Delta_h is the 5-point Laplacian at grid spacing h (App. C's finite
    differences, (f_W + f_E + f_S + f_N - 4 f) / h^2 in the interior), so a row of L has
    kappa^2 + deg / h^2 on the diagonal and -1 / h^2 per existing neighbour.

    Slot order within a cell factor: the cell itself, then its west (x-1), east (x+1),
    south (y-1) and north (y+1) neighbours, those that exist; for alpha = 4 then the
    diagonal neighbours (x-1, y-1), (x+1, y-1), (x-1, y+1), (x+1, y+1) and the nodes
    (x-2, y), (x+2, y), (x, y-2), (x, y+2), those that exist.
    """
    if not (h > 0.0 and np.isfinite(h)):
        raise ValueError("grid spacing h must be finite and > 0")
    if alpha == 4:
        return _prior_factors_l2(nx, ny, kappa, gamma, h)
    if alpha != 2:
        raise ValueError("alpha must be 2 or 4")
    n = nx * ny
    ii, jj = np.divmod(np.arange(n, dtype=np.int64), nx)
    c = ii * nx + jj
    # slot candidates in order self, W, E, S, N and whether each neighbour exists
    cand = np.stack([c, c - 1, c + 1, c - nx, c + nx], axis=1)
    exists = np.stack([np.ones(n, bool), jj > 0, jj < nx - 1, ii > 0, ii < ny - 1], axis=1)
    deg = exists[:, 1:].sum(axis=1)
    coefs = np.empty((n, 5))
    coefs[:, 0] = kappa * kappa + deg / (h * h)
    coefs[:, 1:] = -1.0 / (h * h)
    counts = exists.sum(axis=1)
    ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    return FactorList(n, ptr, cand[exists].astype(np.int64), coefs[exists].astype(np.float64),
                      np.full(n, float(gamma)), np.zeros(n))


def _prior_factors_l2(nx: int, ny: int, kappa: float, gamma: float, h: float = 1.0) -> FactorList:
    """Rows of L^2: L assembled from the alpha = 2 factor rows, squared by a sparse matrix
    product (a library step), each row read out in the slot order of ``_L2_OFFSETS``."""
    import scipy.sparse as sp
    fl1 = prior_factors(nx, ny, kappa, 1.0, 2, h)
    rows = np.repeat(np.arange(fl1.nf), np.diff(fl1.ptr))
    L = sp.csr_matrix((fl1.coef, (rows, fl1.var)), shape=(fl1.n, fl1.n))
    L2 = (L @ L).tocsr()
    n = nx * ny
    ii, jj = np.divmod(np.arange(n, dtype=np.int64), nx)
    cand, exists = [], []
    for dx, dy in _L2_OFFSETS:
        x, y = jj + dx, ii + dy
        cand.append(y * nx + x)
        exists.append((x >= 0) & (x < nx) & (y >= 0) & (y < ny))
    cand = np.stack(cand, axis=1)
    exists = np.stack(exists, axis=1)
    var = cand[exists].astype(np.int64)
    cell = np.repeat(np.arange(n), exists.sum(axis=1))
    coef = np.asarray(L2[cell, var]).reshape(-1).astype(np.float64)
    ptr = np.zeros(n + 1, np.int64)
    np.cumsum(exists.sum(axis=1), out=ptr[1:])
    # the slots are exactly the nonzeros of each row of L^2
    assert L2.nnz == var.size and np.all(coef != 0.0)
    return FactorList(n, ptr, var, coef, np.full(n, float(gamma)), np.zeros(n))


def bilinear_base_weights(nx: int, ny: int, ox: np.ndarray, oy: np.ndarray):
    """Base node (i0, j0) and the four bilinear weights of each location.

    j0 = min(floor(u), nx-2), i0 = min(floor(v), ny-2), fu = u - j0, fv = v - i0; the
    weights on (i0,j0), (i0,j0+1), (i0+1,j0), (i0+1,j0+1) are (1-fu)(1-fv), fu(1-fv),
    (1-fu)fv, fu fv.  Locations must lie in [0, nx-1] x [0, ny-1].
    """
    ox = np.asarray(ox, np.float64)
    oy = np.asarray(oy, np.float64)
    if np.any(ox < 0) or np.any(ox > nx - 1) or np.any(oy < 0) or np.any(oy > ny - 1):
        raise ValueError("observation outside the grid")
    j0 = np.minimum(np.floor(ox), nx - 2).astype(np.int64)
    i0 = np.minimum(np.floor(oy), ny - 2).astype(np.int64)
    fu = ox - j0
    fv = oy - i0
    w = np.stack([(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv], axis=1)
    return i0, j0, w


def obs_factors(nx: int, ny: int, ox, oy, y, noise_var) -> FactorList:
    """One 4-slot factor per observation (slots in the order of the bilinear weights)."""
    m = len(ox)
    n = nx * ny
    if m == 0:
        return FactorList(n, np.zeros(1, np.int64), np.zeros(0, np.int64), np.zeros(0),
                          np.zeros(0), np.zeros(0))
    if nx < 2 or ny < 2:
        raise ValueError("observations need a grid of at least 2 x 2")
    i0, j0, w = bilinear_base_weights(nx, ny, ox, oy)
    b = i0 * nx + j0
    var = np.stack([b, b + 1, b + nx, b + nx + 1], axis=1).reshape(-1)
    nv = np.asarray(noise_var, np.float64)
    if np.any(~(nv > 0)):
        raise ValueError("noise variances must be positive")
    return FactorList(n, np.arange(0, 4 * m + 1, 4, dtype=np.int64), var.astype(np.int64),
                      w.reshape(-1).copy(), 1.0 / nv, np.asarray(y, np.float64).copy())


def with_prior_mean(fl: FactorList, prior_mean) -> FactorList:
    """The cell factors of a prior with mean f_b (Sec. 2.2: the prior N(f_b, Sigma)): factor c
    becomes exp(-(s/2)(a_c . f - a_c . f_b)^2), i.e. its target is r_c = a_c . f_b, written out
    here as the dot product of the factor's coefficients with f_b at its variables."""
    fb = np.asarray(prior_mean, np.float64).reshape(-1)
    if fb.shape[0] != fl.n:
        raise ValueError("prior mean must have one value per node")
    r = np.zeros(fl.nf)
    for f in range(fl.nf):
        sl = slice(fl.ptr[f], fl.ptr[f + 1])
        r[f] = float(np.dot(fl.coef[sl], fb[fl.var[sl]]))
    return FactorList(fl.n, fl.ptr, fl.var, fl.coef, fl.s, r)


def build_factors(nx, ny, kappa, ox, oy, y, noise_var, gamma: float = 1.0, alpha: int = 2,
                  prior_mean=None, h: float = 1.0) -> FactorList:
    """The posterior's factor list: prior cell factors first, then observations in input order.
    ``prior_mean`` (one value per node) gives the cell factors their targets (``with_prior_mean``);
    ``h`` is the grid spacing of the prior's Laplacian (observation locations stay in grid units)."""
    pf = prior_factors(nx, ny, kappa, gamma, alpha, h)
    if prior_mean is not None:
        pf = with_prior_mean(pf, prior_mean)
    return concat(pf, obs_factors(nx, ny, ox, oy, y, noise_var)).check()


def factor_update(a, s, r, lam_c, eta_c):
    """Messages of one factor given its slots' cavities (see ``orc_factor_update``)."""
    a = np.ascontiguousarray(a, np.float64)
    lam_c = np.ascontiguousarray(lam_c, np.float64)
    eta_c = np.ascontiguousarray(eta_c, np.float64)
    k = a.shape[0]
    lo = np.zeros(k)
    eo = np.zeros(k)
    lib().orc_factor_update(k, _p(a, _f64p), float(s), float(r), _p(lam_c, _f64p),
                            _p(eta_c, _f64p), _p(lo, _f64p), _p(eo, _f64p))
    return lo, eo


def init_messages(fl: FactorList, mode: str = "cold", mu0=None, lam0=None):
    """Initial (eta, Lambda) per slot: 'cold', 'paper' or 'warm' (needs mu0, lam0)."""
    code = {"cold": 0, "paper": 1, "warm": 2}[mode]
    me = np.zeros(fl.ne)
    ml = np.zeros(fl.ne)
    if code == 2:
        mu0 = np.ascontiguousarray(mu0, np.float64).reshape(-1)
        lam0 = np.ascontiguousarray(lam0, np.float64).reshape(-1)
    else:
        mu0 = np.zeros(1)
        lam0 = np.zeros(1)
    rc = lib().orc_init_messages(code, fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p),
                                 _p(fl.coef, _f64p), _p(fl.s, _f64p), _p(mu0, _f64p),
                                 _p(lam0, _f64p), _p(me, _f64p), _p(ml, _f64p))
    if rc != 0:
        raise RuntimeError(f"orc_init_messages failed ({rc})")
    return me, ml


def beliefs(fl: FactorList, me, ml):
    be = np.zeros(fl.n)
    bl = np.zeros(fl.n)
    me = np.ascontiguousarray(me, np.float64)
    ml = np.ascontiguousarray(ml, np.float64)
    lib().orc_beliefs(fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(me, _f64p),
                      _p(ml, _f64p), _p(be, _f64p), _p(bl, _f64p))
    return be, bl


def gabp(fl: FactorList, beta: float, iters: int, *, init: str = "cold", mu0=None, lam0=None,
         messages=None):
    """Run ``iters`` synchronous damped iterations.

    Returns ``(mean, var, (msg_eta, msg_lam))``: the marginals mu = eta/Lambda and
    sigma^2 = 1/Lambda (App. A, marginal extraction with c = 1 and no separate unary term)
    and the final messages.  ``messages`` overrides the initialisation.
    """
    if messages is not None:
        me = np.array(messages[0], np.float64, copy=True)
        ml = np.array(messages[1], np.float64, copy=True)
    else:
        me, ml = init_messages(fl, init, mu0, lam0)
    be = np.zeros(fl.n)
    bl = np.zeros(fl.n)
    rc = lib().orc_gabp_run(fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(fl.coef, _f64p),
                            _p(fl.s, _f64p), _p(fl.r, _f64p), float(beta), int(iters),
                            _p(me, _f64p), _p(ml, _f64p), _p(be, _f64p), _p(bl, _f64p))
    if rc != 0:
        raise RuntimeError(f"orc_gabp_run failed ({rc})")
    with np.errstate(divide="ignore", invalid="ignore"):
        return be / bl, 1.0 / bl, (me, ml)


def apply_A(fl: FactorList, x):
    x = np.ascontiguousarray(x, np.float64).reshape(-1)
    out = np.zeros(fl.n)
    lib().orc_apply_A(fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(fl.coef, _f64p),
                      _p(fl.s, _f64p), _p(x, _f64p), _p(out, _f64p))
    return out


def rhs(fl: FactorList):
    out = np.zeros(fl.n)
    lib().orc_rhs(fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(fl.coef, _f64p),
                  _p(fl.s, _f64p), _p(fl.r, _f64p), _p(out, _f64p))
    return out


def residual(fl: FactorList, mu) -> float:
    """Relative residual ||b - A mu||_2 / ||b||_2 in FP64."""
    b = rhs(fl)
    return float(np.linalg.norm(b - apply_A(fl, mu)) / np.linalg.norm(b))


def dense_A(fl: FactorList) -> np.ndarray:
    A = np.zeros((fl.n, fl.n))
    for f in range(fl.nf):
        sl = slice(fl.ptr[f], fl.ptr[f + 1])
        v, a = fl.var[sl], fl.coef[sl]
        A[np.ix_(v, v)] += fl.s[f] * np.outer(a, a)
    return A


def exact_mean(fl: FactorList, nx: int, method: str = "band") -> np.ndarray:
    """Exact posterior mean A^-1 b.

    'band': banded Cholesky in natural order with the factor list's half bandwidth (C);
    'sparse': scipy's sparse LU (a library solve step) for grids too large for the band.
    """
    b = rhs(fl)
    if method == "band":
        return band_solve(fl, nx, b)
    if method == "sparse":
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        rows, cols, vals = [], [], []
        k = np.diff(fl.ptr)
        for kk in np.unique(k):
            fs = np.nonzero(k == kk)[0]
            idx = fl.ptr[fs][:, None] + np.arange(kk)[None, :]
            v = fl.var[idx]
            a = fl.coef[idx] * np.sqrt(fl.s[fs])[:, None]
            rows.append(np.repeat(v, kk, axis=1).reshape(-1))
            cols.append(np.tile(v, (1, kk)).reshape(-1))
            vals.append((a[:, :, None] * a[:, None, :]).reshape(-1))
        A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(fl.n, fl.n))
        return spl.spsolve(A, b)
    raise ValueError(method)


def half_bandwidth(fl: FactorList) -> int:
    """Largest index distance between two variables of one factor: A = sum s a a^T is zero
    farther from the diagonal (2 nx for the alpha = 2 prior, 4 nx for alpha = 4)."""
    k = np.diff(fl.ptr)
    hb = 0
    for kk in np.unique(k):
        if kk == 0:
            continue
        fs = np.nonzero(k == kk)[0]
        v = fl.var[fl.ptr[fs][:, None] + np.arange(kk)[None, :]]
        hb = max(hb, int((v.max(axis=1) - v.min(axis=1)).max()))
    return hb


def band_solve(fl: FactorList, nx: int, b) -> np.ndarray:
    """Solve A x = b (A from the factor list) by the banded Cholesky; the half bandwidth is
    the factor list's (at least 2 nx)."""
    x = np.array(b, np.float64, copy=True).reshape(-1)
    hb = max(2 * nx, half_bandwidth(fl))
    rc = lib().orc_band_solve(fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p),
                              _p(fl.coef, _f64p), _p(fl.s, _f64p), hb, _p(x, _f64p))
    if rc != 0:
        raise RuntimeError(f"orc_band_solve failed ({rc})")
    return x


def exact_variances(fl: FactorList) -> np.ndarray:
    """diag(A^-1) by a dense inverse (small grids only)."""
    if fl.n > 5000:
        raise ValueError("dense variances only for n <= 5000")
    return np.diag(np.linalg.inv(dense_A(fl))).copy()
