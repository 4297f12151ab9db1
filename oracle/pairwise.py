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

Alg. 2 in full ("Re-weighted message passing with multigrid, damping, and early stopping"):
``run_early_stop`` iterates one level under the early-stopping rule of App. B (the reading of
the rank-1 form: reference = mean change between iterations 1 and 2 of the run, stop after the
first t >= 3 whose change is below tau times it), ``upscale`` initialises a finer level's
edge values from the coarser level's ("Upscale Messages"), and ``multigrid`` runs the levels
from the coarsest to the target grid.  Level k has spacing 2^k (kappa_k = 2^k kappa,
gamma_k = gamma / 4^k, the multigrid reading of the rank-1 form), and an observation at a grid
point enters level k only where its location coincides with a level-k grid point (the
paper's rule; grid-point observations only).
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


def run(P, h, c: float, eta: float, iters: int, messages=None, E=None):
    """``iters`` synchronous damped iterations; returns (mean, precision, (a, b), finite).
    Mean and precision are the marginal formulas of App. A with the current messages.
    ``E``: the result of ``edges(P)``, if already computed."""
    n = P.shape[0]
    src, dst, pij, rev = edges(P) if E is None else E
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


def message_change(new, old) -> float:
    """mean |m_new - m_old| over both components of every directed edge."""
    da = np.abs(np.asarray(new[0]) - np.asarray(old[0]))
    db = np.abs(np.asarray(new[1]) - np.asarray(old[1]))
    return float((da.sum() + db.sum()) / (da.size + db.size))


def run_early_stop(P, h, c: float, eta: float, tau: float, max_iters: int, messages=None, ref=None,
                   out_ref=None):
    """Iterate one level under the early-stopping rule (App. B).  Returns (t, mean, precision,
    messages, finite): t = the stopping iteration (None if max_iters came first or the run
    stopped being finite).  The reference change is mean |m_2 - m_1| of this run's first two
    iterations, or ``ref`` when given; ``out_ref`` (a list) receives the reference used."""
    E = edges(P)
    msg = messages if messages is not None else (np.zeros(E[0].size), np.zeros(E[0].size))
    _, _, m1, ok1 = run(P, h, c, eta, 1, messages=msg, E=E)
    mean, prec, m2, ok2 = run(P, h, c, eta, 1, messages=m1, E=E)
    if not (ok1 and ok2):
        return None, mean, prec, m2, False
    if ref is None:
        ref = message_change(m2, m1)
    if out_ref is not None:
        out_ref.append(ref)
    t, cur = 2, m2
    while t < max_iters:
        prev = cur
        mean, prec, cur, ok = run(P, h, c, eta, 1, messages=prev, E=E)
        t += 1
        if not ok:
            return None, mean, prec, cur, False
        if message_change(cur, prev) < tau * ref:
            return t, mean, prec, cur, True
    return None, mean, prec, cur, True


def upscale(msg_c, Pc, nxc: int, nyc: int, Pf, nxf: int, nyf: int):
    """Edge values of the finer level from the coarser level's ("Upscale Messages"): the
    message on the fine edge from node v towards v + o takes the value of the coarse edge
    from v's parent (floor(i/2), floor(j/2)) towards parent + o, or 0 where that coarse edge
    does not exist."""
    sc, dc, _, _ = edges(Pc)
    sf, df, _, _ = edges(Pf)
    fy, fx = np.divmod(sf, nxf)
    ty, tx = np.divmod(df, nxf)
    dy, dx = ty - fy, tx - fx
    py = np.minimum(fy // 2, nyc - 1)
    px = np.minimum(fx // 2, nxc - 1)
    qy, qx = py + dy, px + dx
    inside = (qx >= 0) & (qx < nxc) & (qy >= 0) & (qy < nyc)
    nc = nxc * nyc
    keys = dc.astype(np.int64) * nc + sc          # edges() sorts by (dst, src)
    want = (qy * nxc + qx).astype(np.int64) * nc + (py * nxc + px)
    pos = np.minimum(np.searchsorted(keys, want), keys.size - 1)
    found = inside & (keys[pos] == want)
    a = np.where(found, np.asarray(msg_c[0])[pos], 0.0)
    b = np.where(found, np.asarray(msg_c[1])[pos], 0.0)
    return a, b


def level_observations(ox, oy, y, noise_var, k: int):
    """The grid-point observations that coincide with level-k grid points, in level-k
    coordinates."""
    s = 1 << k
    ox = np.asarray(ox, np.float64)
    oy = np.asarray(oy, np.float64)
    if np.any(ox != np.round(ox)) or np.any(oy != np.round(oy)):
        raise ValueError("the paper's multigrid rule is for grid-point observations")
    sel = (np.mod(ox, s) == 0) & (np.mod(oy, s) == 0)
    return ox[sel] / s, oy[sel] / s, np.asarray(y)[sel], np.asarray(noise_var)[sel]


def multigrid(nx, ny, kappa, gamma, ox, oy, y, noise_var, levels: int, c: float, eta: float, tau: float,
              max_iters: int, reference: str = "level"):
    """Alg. 2: levels - 1 coarse levels and the target, each iterated under the early-stopping
    rule from the upscaled edge values of the level below it (zero on the coarsest).  Returns
    (mean, precision, stop) on the target grid, stop[k] = the stopping iteration of level k.

    ``reference`` reads which m_1, m_2 the rule compares against (App. B writes them without a
    level): "level" = the first two iterations of each level (the reading the library follows),
    "first" = those of the first, coarsest level, for every level."""
    if reference not in ("level", "first"):
        raise ValueError(reference)
    prev = None
    stop = {}
    mean = prec = None
    first_ref = []
    for k in range(levels - 1, -1, -1):
        s = 1 << k
        nxk, nyk = -(-nx // s), -(-ny // s)
        lox, loy, ly, lv = level_observations(ox, oy, y, noise_var, k)
        from . import build_factors
        fl = build_factors(nxk, nyk, kappa * s, lox, loy, ly, lv, gamma=gamma / (s * s))
        P, h = assemble(fl)
        msg = None if prev is None else upscale(prev[0], prev[1], prev[2], prev[3], P, nxk, nyk)
        ref = first_ref[0] if (reference == "first" and first_ref) else None
        t, mean, prec, msg, ok = run_early_stop(P, h, c, eta, tau, max_iters, msg, ref=ref,
                                                out_ref=first_ref if not first_ref else None)
        stop[k] = t
        prev = (msg, P, nxk, nyk)
    return mean, prec, stop
