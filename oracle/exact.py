"""Exact posterior solves for grids too large for the banded Cholesky.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only the tests, the smoke check, the
benchmark's CPU-baseline leg and the committed scripts that write stored expected values may
use it.  It shares no code with the CUDA library.

The posterior of the paper (Sec. 2.1 problem statement; Sec. 3.1 prior P = gamma L^T L; Sec. 3.2
observations) is N(A^-1 b, A^-1) with A = gamma L^T L + H^T R^-1 H and b = H^T R^-1 y.  Loopy
GaBP means, once converged, equal A^-1 b (Sec. 2.3, the Weiss-Freeman result the paper cites),
so A^-1 b is what the GPU's converged means are judged against.

* ``exact_mean_pcg``: A^-1 b by the preconditioned conjugate gradient method (Hestenes and
  Stiefel), in FP64, to ||b - A x|| / ||b|| <= tol (default 1e-13).  The preconditioner is one
  symmetric multigrid V-cycle: Galerkin coarse operators P^T A P with bilinear prolongation P
  (built by sparse matrix products, a library step), forward Gauss-Seidel sweeps before and
  backward sweeps after each coarse correction, and an exact sparse LU solve on the coarsest
  grid.  The preconditioner only sets how fast the iteration gets there: the answer is A^-1 b
  to the tolerance whatever it is.  ``precond="dct"`` is the other preconditioner of this
  module: the exact inverse of the prior precision gamma L^T L through the 2-D DCT-II, where
  L = kappa^2 I + graph Laplacian (zero-Neumann) is diagonal with eigenvalues
  kappa^2 + 4 sin^2(pi k / 2 nx) + 4 sin^2(pi l / 2 ny).  It is exact without observations
  and takes thousands of iterations with the workloads' dense, precise observations (9,198 to
  1e-13 on the 256^2 track case, against 41 with the V-cycle), so it serves small cases and
  checks.
* ``prior_covariance_column``: column k of (gamma L^T L)^-1 through the same DCT (a closed
  form used by the single-observation check).
* ``exact_variances_band``: diag(A^-1) by selected inversion on the band (C).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import FactorList, _f64p, _i64p, _p, half_bandwidth, lib, rhs

__all__ = ["assemble_csr", "mg_hierarchy", "exact_mean_pcg", "dct_prior_solve",
           "prior_covariance_column", "exact_variances_band"]


def _clib():
    L = lib()
    if not hasattr(L, "_exact_ready"):
        L.orc_assemble_csr.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p,
                                       _i64p, _i64p, _i64p, _f64p]
        L.orc_assemble_csr.restype = ctypes.c_int
        L.orc_gs_sweep.argtypes = [ctypes.c_int64, _i64p, _i64p, _f64p, _f64p, _f64p, ctypes.c_int,
                                   ctypes.c_int]
        L.orc_gs_sweep.restype = ctypes.c_int
        L.orc_band_selinv.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p,
                                      ctypes.c_int64, _f64p]
        L.orc_band_selinv.restype = ctypes.c_int
        L._exact_ready = True
    return L


class _CSR:
    """A CSR matrix with int64 indices, as the C sweeps take it, plus its scipy view."""

    def __init__(self, m):
        import scipy.sparse as sp
        m = sp.csr_matrix(m)
        m.sort_indices()
        self.n = m.shape[0]
        self.rp = np.ascontiguousarray(m.indptr, np.int64)
        self.ci = np.ascontiguousarray(m.indices, np.int64)
        self.val = np.ascontiguousarray(m.data, np.float64)
        self.sp = m

    def gs(self, b, x, backward: bool, sweeps: int):
        rc = _clib().orc_gs_sweep(self.n, _p(self.rp, _i64p), _p(self.ci, _i64p), _p(self.val, _f64p),
                                  _p(b, _f64p), _p(x, _f64p), int(backward), int(sweeps))
        if rc != 0:
            raise RuntimeError("Gauss-Seidel sweep met a non-positive diagonal")


def assemble_csr(fl: FactorList):
    """A = sum_f s_f a_f a_f^T as a scipy CSR matrix (assembled row by row in C)."""
    import scipy.sparse as sp
    L = _clib()
    n = fl.n
    row_len = np.zeros(n, np.int64)
    rc = L.orc_assemble_csr(n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(fl.coef, _f64p),
                            _p(fl.s, _f64p), _p(row_len, _i64p), None, None, None)
    if rc != 0:
        raise RuntimeError(f"orc_assemble_csr (count) failed ({rc})")
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(row_len, out=rp[1:])
    ci = np.zeros(int(rp[-1]), np.int64)
    val = np.zeros(int(rp[-1]))
    rc = L.orc_assemble_csr(n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(fl.coef, _f64p),
                            _p(fl.s, _f64p), _p(row_len, _i64p), _p(rp, _i64p), _p(ci, _i64p),
                            _p(val, _f64p))
    if rc != 0:
        raise RuntimeError(f"orc_assemble_csr (fill) failed ({rc})")
    return sp.csr_matrix((val, ci, rp), shape=(n, n))


def _interp_1d(nf: int):
    """Linear interpolation from ceil(nf/2) coarse points (at the even fine points) to nf fine
    points: an odd fine point takes the mean of its two coarse neighbours, or the one it has."""
    import scipy.sparse as sp
    nc = (nf + 1) // 2
    rows, cols, vals = [], [], []
    for i in range(nf):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        elif (i + 1) // 2 < nc:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
        else:
            rows.append(i); cols.append((i - 1) // 2); vals.append(1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def mg_hierarchy(A, nx: int, ny: int, coarsest: int = 64):
    """Galerkin levels: A_0 = A, A_{l+1} = P_l^T A_l P_l with P_l = P_y (x) P_x (bilinear), halving
    both axes until the larger side is at most ``coarsest``; the coarsest level is LU-factored."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    levels = [_CSR(A)]
    Ps = []
    cur = levels[0].sp
    while max(nx, ny) > coarsest and min(nx, ny) > 2:
        Px, Py = _interp_1d(nx), _interp_1d(ny)
        P = sp.kron(Py, Px, format="csr")
        cur = (P.T @ cur @ P).tocsr()
        nx, ny = Px.shape[1], Py.shape[1]
        Ps.append(P)
        levels.append(_CSR(cur))
    lu = spl.splu(levels[-1].sp.tocsc())
    return levels, Ps, lu


def _vcycle(levels, Ps, lu, l: int, b: np.ndarray, nu: int) -> np.ndarray:
    if l == len(levels) - 1:
        return lu.solve(b)
    M = levels[l]
    x = np.zeros_like(b)
    M.gs(b, x, backward=False, sweeps=nu)
    r = b - M.sp @ x
    x += Ps[l] @ _vcycle(levels, Ps, lu, l + 1, np.ascontiguousarray(Ps[l].T @ r), nu)
    M.gs(b, x, backward=True, sweeps=nu)
    return x


def dct_prior_solve(v: np.ndarray, nx: int, ny: int, kappa: float, gamma: float = 1.0) -> np.ndarray:
    """(gamma L^T L)^-1 v through the orthonormal 2-D DCT-II (L symmetric, so L^T L = L^2)."""
    from scipy import fft as sfft
    kx = 4.0 * np.sin(np.pi * np.arange(nx) / (2.0 * nx)) ** 2
    ky = 4.0 * np.sin(np.pi * np.arange(ny) / (2.0 * ny)) ** 2
    lam = kappa * kappa + ky[:, None] + kx[None, :]
    c = sfft.dctn(np.asarray(v, np.float64).reshape(ny, nx), type=2, norm="ortho")
    return sfft.idctn(c / (gamma * lam * lam), type=2, norm="ortho").reshape(-1)


def prior_covariance_column(k: int, nx: int, ny: int, kappa: float, gamma: float = 1.0) -> np.ndarray:
    e = np.zeros(nx * ny)
    e[k] = 1.0
    return dct_prior_solve(e, nx, ny, kappa, gamma)


def exact_mean_pcg(fl: FactorList, nx: int, ny: int, *, tol: float = 1e-13, maxit: int = 5000,
                   precond: str = "mg", kappa: float | None = None, gamma: float = 1.0,
                   nu: int = 2, coarsest: int = 64, x0=None, verbose: bool = False):
    """A^-1 b by preconditioned conjugate gradients to ||b - A x|| / ||b|| <= tol.

    Returns ``(x, info)`` with the iteration count and the final relative residual (recomputed
    from the factor list as ||b - A x|| / ||b||, independently of the assembled matrix).
    ``precond``: "mg" (symmetric V-cycle, ``nu`` sweeps each side) or "dct" (exact inverse of
    the prior precision; needs ``kappa`` and ``gamma``).  Raises if tol is not reached."""
    from . import residual
    A = assemble_csr(fl)
    b = rhs(fl)
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return np.zeros(fl.n), {"iterations": 0, "rel_residual": 0.0}
    if precond == "mg":
        levels, Ps, lu = mg_hierarchy(A, nx, ny, coarsest)

        def M(r):
            return _vcycle(levels, Ps, lu, 0, r, nu)
    elif precond == "dct":
        if kappa is None:
            raise ValueError("the DCT preconditioner needs kappa")

        def M(r):
            return dct_prior_solve(r, nx, ny, kappa, gamma)
    else:
        raise ValueError(precond)
    x = np.zeros(fl.n) if x0 is None else np.array(x0, np.float64, copy=True).reshape(-1)
    r = b - A @ x
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    replaced = 0
    rel = float(np.linalg.norm(r)) / nb
    while rel > tol and it < maxit and replaced <= 8:
        Ap = A @ p
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        it += 1
        rel = float(np.linalg.norm(r)) / nb
        if verbose and it % 10 == 0:
            print(f"pcg {it}: {rel:.3e}", flush=True)
        if rel <= tol:
            # the updated residual drifts from b - A x by rounding: replace it by the true one
            # and carry on (restarting the search direction) until the true one is below tol
            r = b - A @ x
            rel = float(np.linalg.norm(r)) / nb
            replaced += 1      # a tolerance below the rounding floor ends after a few of these
            if rel <= tol:
                break
            z = M(r)
            p = z.copy()
            rz = float(r @ z)
            continue
        z = M(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    true_rel = residual(fl, x)
    if not true_rel <= 2.0 * tol:
        raise RuntimeError(f"PCG stopped at relative residual {true_rel:.3e} after {it} iterations")
    return x, {"iterations": it, "rel_residual": true_rel, "precond": precond}


def exact_variances_band(fl: FactorList, nx: int) -> np.ndarray:
    """diag(A^-1) by selected inversion on the band (Takahashi recurrences, C); memory
    2 n (bw + 1) doubles with bw the factor list's half bandwidth (2 nx for alpha = 2)."""
    n = fl.n
    bw = max(2 * nx, half_bandwidth(fl))
    if n * (bw + 1) > 2 ** 27:
        raise ValueError("the band is too large for selected inversion here (n (bw + 1) > 2^27)")
    out = np.zeros(n)
    rc = _clib().orc_band_selinv(n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(fl.coef, _f64p),
                                 _p(fl.s, _f64p), bw, _p(out, _f64p))
    if rc != 0:
        raise RuntimeError(f"orc_band_selinv failed ({rc})")
    return out
