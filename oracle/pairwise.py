"""The paper's pairwise re-weighted Gaussian message passing (TEST INFRASTRUCTURE ONLY).

App. A ("Gaussian Setting", "Re-weighted message updates"; Ruozzi and Tatikonda's scheme):
the posterior N(P^-1 h, P^-1) with P = gamma L^T L + H^T R^-1 H and h = H^T R^-1 y is written
with one node factor exp(-P_ii f_i^2 / 2 + h_i f_i) per node and one pair factor
exp(-P_ij f_i f_j) per nonzero off-diagonal P_ij (the 13-point pattern of L^T L).  Messages are
fractional: m^(1/c) = exp(-a f^2 / 2 + b f) from a pair factor to a variable, and
exp(-alpha f^2 / 2 + beta f) from a variable to a pair factor, with

    alpha_{j->i} = P_jj + c sum_{k != i} a_{kj} + (c - 1) a_{ij},
    beta_{j->i}  = h_j  + c sum_{k != i} b_{kj} + (c - 1) b_{ij},
    a_{ji} = -(P_ij / c)^2 / alpha_{j->i},   b_{ji} = -beta_{j->i} (P_ij / c) / alpha_{j->i},

where (a_{kj}, b_{kj}) is the message from the pair factor of (k, j) to f_j.  The paper prints
b with the opposite sign; this follows the integral that defines the message (the same reading
as for the rank-1 form), with every message in the information convention exp(-a f^2/2 + b f)
(so the marginal is (h_i + c sum_k b_ki) / (P_ii + c sum_k a_ki)).  Damping with the paper's
learning rate eta: m <- (1 - eta) m_old + eta m_new.  Messages start at zero.
"""
from __future__ import annotations

import numpy as np


def assemble(fl):
    """P (scipy CSR, the posterior precision of the factor list) and h (= b, the information)."""
    import scipy.sparse as sp
    from . import rhs
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
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(fl.n, fl.n))
    P.sum_duplicates()
    return P, rhs(fl)


def edges(P):
    """Directed edges e = (src j, dst i) for every nonzero off-diagonal P_ij, the index of the
    reverse edge, and P_ij.  Edge e carries the message of the pair factor of (i, j) to f_i."""
    C = P.tocoo()
    off = C.row != C.col
    dst, src, pij = C.row[off], C.col[off], C.data[off]
    order = np.lexsort((src, dst))
    dst, src, pij = dst[order], src[order], pij[order]
    key = dst.astype(np.int64) * P.shape[0] + src
    rkey = src.astype(np.int64) * P.shape[0] + dst
    rev = np.searchsorted(key, rkey)
    assert np.array_equal(key[rev], rkey)
    return src, dst, pij, rev


def factor_message(alpha, beta, pij, c):
    """(a, b) of the fractional pair-factor message from the variable-to-factor (alpha, beta)."""
    q = pij / c
    return -(q * q) / alpha, -beta * q / alpha


def run(P, h, c: float, eta: float, iters: int, messages=None):
    """``iters`` synchronous damped iterations; returns (mean, precision, (a, b), finite).
    Mean and precision are the marginal formulas of App. A with the current messages."""
    n = P.shape[0]
    src, dst, pij, rev = edges(P)
    Pd = P.diagonal()
    a = np.zeros(src.size) if messages is None else np.array(messages[0], np.float64, copy=True)
    b = np.zeros(src.size) if messages is None else np.array(messages[1], np.float64, copy=True)
    ok = True
    with np.errstate(all="ignore"):
        for _ in range(iters):
            S = np.bincount(dst, a, n)
            T = np.bincount(dst, b, n)
            ar, br = a[rev], b[rev]   # message of the same pair factor to f_src
            alpha = Pd[src] + c * (S[src] - ar) + (c - 1.0) * ar
            beta = h[src] + c * (T[src] - br) + (c - 1.0) * br
            an, bn = factor_message(alpha, beta, pij, c)
            a = (1.0 - eta) * a + eta * an
            b = (1.0 - eta) * b + eta * bn
            if not (np.all(np.isfinite(a)) and np.all(np.isfinite(b))):
                ok = False
                break
        S = np.bincount(dst, a, n)
        T = np.bincount(dst, b, n)
        prec = Pd + c * S
        mean = (h + c * T) / prec
    return mean, prec, (a, b), ok
