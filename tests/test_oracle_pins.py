"""Pins of the CPU oracle to the paper and to the mathematics (not to itself).

Each test ties one part of the oracle to something independent: a closed form, a
dense linear-algebra definition built from the paper's matrices, a textbook special
case, or brute force on tiny inputs.  The comments name the plausible mistake each one
would catch.
"""
import math

import numpy as np
import pytest

import gabp_synth


# ---------------------------------------------------------------------------------------
# Factor-to-variable update (App. A) against the dense Schur complement
# ---------------------------------------------------------------------------------------

def _schur_message(a, s, r, lam_c, eta_c, v):
    """Marginal of x_v of  factor * prod_{u != v} N^-1(eta_u, lam_u), by dense algebra."""
    k = len(a)
    J = s * np.outer(a, a)
    h = s * r * np.asarray(a, float)
    for u in range(k):
        if u != v:
            J[u, u] += lam_c[u]
            h[u] += eta_c[u]
    o = [u for u in range(k) if u != v]
    if not o:
        return J[v, v], h[v]
    Joo = J[np.ix_(o, o)]
    Jvo = J[v, o]
    return J[v, v] - Jvo @ np.linalg.solve(Joo, Jvo), h[v] - Jvo @ np.linalg.solve(Joo, h[o])


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_factor_update_equals_schur_complement(orc, k):
    # catches: wrong leave-one-out set, missing 1/s term, sign of the mean term, a transposed
    # (a_v vs a_u) coefficient
    rng = np.random.default_rng(100 + k)
    for _ in range(50):
        a = rng.normal(size=k) * rng.uniform(0.1, 3.0)
        s = rng.uniform(0.05, 20.0)
        r = rng.normal()
        lam_c = rng.uniform(0.05, 10.0, k)
        eta_c = rng.normal(size=k) * 3
        lo, eo = orc.factor_update(a, s, r, lam_c, eta_c)
        for v in range(k):
            L_ref, E_ref = _schur_message(a, s, r, lam_c, eta_c, v)
            assert lo[v] == pytest.approx(L_ref, rel=1e-11, abs=1e-13)
            assert eo[v] == pytest.approx(E_ref, rel=1e-10, abs=1e-12)


def test_pairwise_factor_reduces_to_paper_update(orc):
    """k = 2: the rank-1 factor splits into the paper's nodewise factors
    phi_i = exp(-P_ii f_i^2 / 2 + h_i f_i) and a pairwise factor exp(-P_ij f_i f_j)
    (App. A, Gaussian setting, non-zero mean).  With the var-to-factor message of f_j
    written exp(-alpha f_j^2 / 2 - beta f_j), alpha = P_jj + (cavity precision of f_j) and
    beta = -h_j - (cavity information of f_j) (App. A, variable-to-factor update with
    non-zero mean).

    Precision: the paper's a_ij = -P_ij^2 / alpha_ij (Eq. for the factor-to-variable update)
    is matched exactly.  Information: the integral that defines the message (App. A,
    factor-to-variable message) gives exp(+(P_ij^2 / 2 alpha) f_i^2 + (beta P_ij / alpha) f_i),
    i.e. b_ij = -beta_ij P_ij / alpha_ij in the paper's exp(-a f^2/2 - b f) form.  The printed
    b_ij = +beta_ij P_ij / alpha_ij comes from completing the square as (f_j - beta/alpha)^2
    where exp(-alpha f^2/2 - beta f) needs (f_j + beta/alpha)^2; we follow the integral.
    Our message also carries the factor's own nodewise part (P_ii, h_i)."""
    rng = np.random.default_rng(7)
    for _ in range(100):
        a = rng.normal(size=2) * 2
        s = rng.uniform(0.1, 5)
        r = rng.normal()
        lam_c = rng.uniform(0.1, 5, 2)
        eta_c = rng.normal(size=2)
        lo, eo = orc.factor_update(a, s, r, lam_c, eta_c)
        for i, j in [(0, 1), (1, 0)]:
            P_ii, P_jj, P_ij = s * a[i] ** 2, s * a[j] ** 2, s * a[i] * a[j]
            h_i, h_j = s * r * a[i], s * r * a[j]
            alpha = P_jj + lam_c[j]
            beta = -h_j - eta_c[j]
            a_paper = -P_ij ** 2 / alpha
            b_integral = -beta * P_ij / alpha
            assert lo[i] == pytest.approx(P_ii + a_paper, rel=1e-11, abs=1e-13)
            # information = -b in the paper's parameterisation
            assert eo[i] == pytest.approx(h_i - b_integral, rel=1e-10, abs=1e-12)
        # the pairwise message itself, by direct numerical integration over f_j
        i, j = 0, 1
        P_ij = s * a[0] * a[1]
        alpha = s * a[1] ** 2 + lam_c[1]
        beta = -s * r * a[1] - eta_c[1]
        fj = np.linspace(-60, 60, 200001)
        def logmsg(fi):
            g = -0.5 * alpha * fj ** 2 - beta * fj - P_ij * fi * fj
            mx = g.max()
            return mx + np.log(np.trapezoid(np.exp(g - mx), fj))
        # fit log m(f_i) = -a f^2/2 - b f + c from three points
        f3 = np.array([-0.5, 0.0, 0.5])
        l3 = np.array([logmsg(x) for x in f3])
        a_num = -(l3[0] - 2 * l3[1] + l3[2]) / 0.25
        b_num = -(l3[2] - l3[0]) / 1.0
        assert a_num == pytest.approx(-P_ij ** 2 / alpha, rel=1e-6, abs=1e-8)
        assert b_num == pytest.approx(-beta * P_ij / alpha, rel=1e-6, abs=1e-8)


def test_zero_precision_cavity_gives_the_limit_message(orc):
    """A cavity of zero precision and finite information is the linear potential exp(eta x):
    the factor's messages are the dense Schur complement with that zero on the diagonal (the
    integral of App. A stays proper along the factor's direction), which the formulas reach
    as the precision tends to zero.  Catches: dropping such a slot's information (a (0, 0)
    message), a wrong sign or a_u / a_v swap in the limit, a jump at the precision floor."""
    a = np.array([2.0, -1.0, -1.0])
    lam = np.array([1.0, 0.0, 2.0])
    eta = np.array([0.1, 0.2, 0.3])
    lo, eo = orc.factor_update(a, 1.0, 0.3, lam, eta)
    for v in range(3):
        L_ref, E_ref = _schur_message(a, 1.0, 0.3, lam, eta, v)
        assert lo[v] == pytest.approx(L_ref, rel=1e-12, abs=1e-18)
        assert eo[v] == pytest.approx(E_ref, rel=1e-12)
    # the other slots' messages: precision 0, information -a_v eta_1 / a_1
    assert abs(lo[0]) < 1e-18 and eo[0] == pytest.approx(0.4) and abs(lo[2]) < 1e-18 and eo[2] == pytest.approx(-0.2)
    # a small positive precision: the dense Schur complement, which tends to the same limit
    for lam1 in (1e-8, 1e-12):
        lam_s = np.array([1.0, lam1, 2.0])
        lo, eo = orc.factor_update(a, 1.0, 0.3, lam_s, eta)
        for v in range(3):
            L_ref, E_ref = _schur_message(a, 1.0, 0.3, lam_s, eta, v)
            assert lo[v] == pytest.approx(L_ref, rel=1e-9) and eo[v] == pytest.approx(E_ref, rel=1e-9)
    # no jump at the floor (1e-20 a_u^2), and a negative cavity is read as a zero one
    lo1, eo1 = orc.factor_update(a, 1.0, 0.3, np.array([1.0, 1.01e-20, 2.0]), eta)
    lo2, eo2 = orc.factor_update(a, 1.0, 0.3, np.array([1.0, 0.99e-20, 2.0]), eta)
    lon, eon = orc.factor_update(a, 1.0, 0.3, np.array([1.0, -1.0, 2.0]), eta)
    assert np.allclose(eo1, eo2, rtol=1e-12, atol=0) and np.allclose(eon, eo2, rtol=1e-12, atol=0)
    assert np.all(np.isfinite(lon)) and np.all(np.isfinite(eon))
    # two such slots: the limit along precisions shrinking as c a_u^2 (dense Schur at c = 1e-9)
    a4 = np.array([2.0, -1.0, -0.5, 0.25])
    eta4 = np.array([0.1, 0.2, -0.6, 0.3])
    lo, eo = orc.factor_update(a4, 1.0, 0.3, np.array([1.0, 0.0, 0.0, 3.0]), eta4)
    lam_c = np.array([1.0, 1e-9 * a4[1] ** 2, 1e-9 * a4[2] ** 2, 3.0])
    for v in range(4):
        L_ref, E_ref = _schur_message(a4, 1.0, 0.3, lam_c, eta4, v)
        assert eo[v] == pytest.approx(E_ref, rel=1e-6, abs=1e-12) and lo[v] == pytest.approx(L_ref, rel=1e-6, abs=1e-8)
    # zero coefficients are skipped even when the cavity is non-positive
    lo, eo = orc.factor_update(np.array([1.0, 0.0]), 2.0, 0.5, np.array([1.0, -1.0]),
                               np.array([0.0, 0.0]))
    assert lo[0] == pytest.approx(2.0) and eo[0] == pytest.approx(1.0)
    assert lo[1] == 0 and eo[1] == 0


# ---------------------------------------------------------------------------------------
# Factor graph construction against the paper's matrices, built densely and independently
# ---------------------------------------------------------------------------------------

def _dense_L(nx, ny, kappa):
    """kappa^2 I - Delta_h with the zero-Neumann (cell-centred ghost) boundary, from the
    finite-difference definition: -Delta_h f_i = sum over existing neighbours (f_i - f_j)."""
    n = nx * ny
    L = kappa ** 2 * np.eye(n)
    for i in range(ny):
        for j in range(nx):
            c = i * nx + j
            for di, dj in [(0, -1), (0, 1), (-1, 0), (1, 0)]:
                ii, jj = i + di, j + dj
                if 0 <= ii < ny and 0 <= jj < nx:
                    L[c, c] += 1.0
                    L[c, ii * nx + jj] -= 1.0
    return L


def _dense_H(nx, ny, ox, oy):
    """Bilinear interpolation rows, written as 'interpolate the unit vectors'."""
    m = len(ox)
    H = np.zeros((m, nx * ny))
    for k in range(m):
        u, v = ox[k], oy[k]
        for i in range(ny):
            for j in range(nx):
                # tent functions: weight of node (i, j) at (u, v)
                wx = max(0.0, 1.0 - abs(u - j))
                wy = max(0.0, 1.0 - abs(v - i))
                H[k, i * nx + j] = wx * wy
    return H


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 2), (5, 7), (8, 6)])
def test_factor_list_matches_dense_posterior(orc, nx, ny):
    # catches: wrong boundary degree, a dropped neighbour, wrong bilinear corner order, H^T vs H
    rng = np.random.default_rng(nx * 10 + ny)
    kappa = 0.37
    m = 9
    ox = rng.uniform(0, nx - 1, m)
    oy = rng.uniform(0, ny - 1, m)
    ox[0], oy[0] = nx - 1, ny - 1          # far corner: clamped into the last cell, fu = fv = 1
    ox[1], oy[1] = 0.0, 0.0
    y = rng.normal(size=m)
    nv = rng.uniform(0.01, 0.2, m)
    fl = orc.build_factors(nx, ny, kappa, ox, oy, y, nv)
    L = _dense_L(nx, ny, kappa)
    H = _dense_H(nx, ny, ox, oy)
    Rinv = np.diag(1.0 / nv)
    A = L.T @ L + H.T @ Rinv @ H
    b = H.T @ Rinv @ y
    np.testing.assert_allclose(orc.dense_A(fl), A, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(orc.rhs(fl), b, rtol=1e-13, atol=1e-12)
    x = rng.normal(size=nx * ny)
    np.testing.assert_allclose(orc.apply_A(fl, x), A @ x, rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(orc.exact_mean(fl, nx), np.linalg.solve(A, b), rtol=1e-10, atol=1e-11)


def test_bilinear_weights_reproduce_linear_functions(orc):
    # catches: swapped fu/fv, off-by-one clamp, weights not summing to one
    nx, ny = 9, 5
    rng = np.random.default_rng(3)
    ox = np.concatenate([rng.uniform(0, nx - 1, 200), [nx - 1, 0, nx - 1, 3.0]])
    oy = np.concatenate([rng.uniform(0, ny - 1, 200), [ny - 1, ny - 1, 0, 2.0]])
    i0, j0, w = orc.bilinear_base_weights(nx, ny, ox, oy)
    assert np.all(j0 <= nx - 2) and np.all(i0 <= ny - 2) and np.all(w >= -1e-15)
    np.testing.assert_allclose(w.sum(1), 1.0, rtol=0, atol=1e-14)
    f = lambda x, y: 0.3 + 1.7 * x - 2.1 * y  # noqa: E731
    vals = (w[:, 0] * f(j0, i0) + w[:, 1] * f(j0 + 1, i0) + w[:, 2] * f(j0, i0 + 1)
            + w[:, 3] * f(j0 + 1, i0 + 1))
    np.testing.assert_allclose(vals, f(ox, oy), rtol=0, atol=1e-12)
    # the far edge goes into the last cell with the full weight on the far node
    assert j0[-4] == nx - 2 and i0[-4] == ny - 2 and w[-4, 3] == 1.0
    # an integer location puts weight 1 on its node
    assert j0[-1] == 3 and i0[-1] == 2 and w[-1, 0] == 1.0
    with pytest.raises(ValueError):
        orc.bilinear_base_weights(nx, ny, np.array([nx - 1 + 1e-9]), np.array([0.0]))
    with pytest.raises(ValueError):
        orc.bilinear_base_weights(nx, ny, np.array([0.0]), np.array([-1e-12]))


# ---------------------------------------------------------------------------------------
# Closed forms: the DCT diagonalises L under zero-Neumann
# ---------------------------------------------------------------------------------------

def _dct_basis(nx, ny, k, l):
    from scipy import fft as sfft
    e = np.zeros((ny, nx))
    e[l, k] = 1.0
    return sfft.idctn(e, type=2, norm="ortho").reshape(-1)


def test_prior_precision_eigenvectors_are_dct(orc):
    # catches: a non-symmetric boundary (reflect ghost), wrong diagonal, missing gamma
    nx, ny, kappa, gamma = 12, 9, 0.21, 1.7
    fl = orc.prior_factors(nx, ny, kappa, gamma)
    lam = gabp_synth.neumann_eigenvalues(nx, ny, kappa)
    for (k, l) in [(0, 0), (1, 0), (0, 1), (5, 3), (11, 8), (7, 2)]:
        phi = _dct_basis(nx, ny, k, l)
        np.testing.assert_allclose(orc.apply_A(fl, phi), gamma * lam[l, k] ** 2 * phi, rtol=0,
                                   atol=1e-11)
    # closed form of the eigenvalues (independent of the synth helper)
    assert lam[0, 0] == pytest.approx(kappa ** 2)
    assert lam[ny - 1, nx - 1] == pytest.approx(
        kappa ** 2 + 4 * math.sin(math.pi * (nx - 1) / (2 * nx)) ** 2
        + 4 * math.sin(math.pi * (ny - 1) / (2 * ny)) ** 2)


@pytest.mark.parametrize("alpha", [2, 4])
def test_grid_spacing_scales_the_laplacian(orc, alpha):
    # catches: h applied to kappa instead of the Laplacian, h instead of h^2, the diagonal's
    # degree term left unscaled.  On the DCT basis the operator at spacing h has eigenvalue
    # kappa^2 + (4 / h^2) (sin^2(pi k / 2 nx) + sin^2(pi l / 2 ny)) (its precision that to the
    # power alpha, times gamma), and on the unit interval the first mode tends to the
    # continuum Neumann eigenvalue kappa^2 + pi^2 as h -> 0.
    nx, ny, kappa, gamma, h = 10, 7, 1.3, 0.8, 0.25
    fl = orc.prior_factors(nx, ny, kappa, gamma, alpha, h)
    for (k, l) in [(0, 0), (1, 0), (0, 1), (4, 3), (9, 6)]:
        phi = _dct_basis(nx, ny, k, l)
        ev = kappa ** 2 + (4.0 / h ** 2) * (math.sin(math.pi * k / (2 * nx)) ** 2 + math.sin(math.pi * l / (2 * ny)) ** 2)
        np.testing.assert_allclose(orc.apply_A(fl, phi), gamma * ev ** alpha * phi, rtol=1e-12,
                                   atol=1e-9 * ev ** alpha)
    # h = 1 is the unit-spacing operator
    f1, f0 = orc.prior_factors(6, 5, kappa, gamma, alpha, 1.0), orc.prior_factors(6, 5, kappa, gamma, alpha)
    assert np.array_equal(f1.coef, f0.coef) and np.array_equal(f1.var, f0.var)
    # continuum: first Neumann mode of the unit square's x direction, nx = 1 / h nodes
    for n1 in (64, 256):
        hh = 1.0 / n1
        fl = orc.prior_factors(n1, 2, kappa, 1.0, 2, hh)
        phi = _dct_basis(n1, 2, 1, 0)
        ev = float(phi @ orc.apply_A(fl, phi)) ** 0.5   # P = L^2: sqrt of the Rayleigh quotient
        assert ev == pytest.approx(kappa ** 2 + math.pi ** 2, rel=2.0 / n1 ** 2)


def test_band_solver_matches_dct_solve(orc):
    from scipy import fft as sfft
    nx, ny, kappa = 24, 17, 0.15
    fl = orc.prior_factors(nx, ny, kappa)
    rng = np.random.default_rng(5)
    b = rng.normal(size=(ny, nx))
    lam = gabp_synth.neumann_eigenvalues(nx, ny, kappa)
    x_dct = sfft.idctn(sfft.dctn(b, type=2, norm="ortho") / lam ** 2, type=2, norm="ortho")
    x = orc.band_solve(fl, nx, b.reshape(-1))
    np.testing.assert_allclose(x, x_dct.reshape(-1), rtol=1e-9, atol=1e-9 * np.abs(x_dct).max())


def test_single_observation_posterior_closed_form(orc):
    """One observation with weight 1 on node i: posterior mean = y Sigma[:, i] / (Sigma_ii + s2),
    with Sigma = (L^T L)^-1 from the DCT (GP regression with one data point, Sec. 2.2)."""
    from scipy import fft as sfft
    nx, ny, kappa = 16, 12, 0.4
    j, i = 5, 7
    yv, s2 = 1.3, 0.05
    fl = orc.build_factors(nx, ny, kappa, np.array([float(j)]), np.array([float(i)]),
                           np.array([yv]), np.array([s2]))
    lam = gabp_synth.neumann_eigenvalues(nx, ny, kappa)
    e = np.zeros((ny, nx))
    e[i, j] = 1.0
    col = sfft.idctn(sfft.dctn(e, type=2, norm="ortho") / lam ** 2, type=2, norm="ortho").reshape(-1)
    expect = yv * col / (col[i * nx + j] + s2)
    np.testing.assert_allclose(orc.exact_mean(fl, nx), expect, rtol=1e-10, atol=1e-12)
    mu, _, _ = orc.gabp(fl, 0.5, 3000)
    np.testing.assert_allclose(mu, expect, rtol=1e-8, atol=1e-10 * np.abs(expect).max())


# ---------------------------------------------------------------------------------------
# Message passing: trees are exact (App. A), loopy fixed points are the exact mean
# ---------------------------------------------------------------------------------------

def _random_tree_factors(orc, rng, n_target=30):
    """A tree-structured factor graph: each new factor joins one existing variable with
    1-4 new ones; every variable also gets a unary factor so the precision is SPD."""
    var_lists, coefs, ss, rs = [], [], [], []
    n = 1
    while n < n_target:
        k_new = int(rng.integers(1, 5))
        anchor = int(rng.integers(0, n))
        vs = [anchor] + list(range(n, n + k_new))
        n += k_new
        var_lists.append(vs)
        coefs.append(rng.normal(size=len(vs)))
        ss.append(rng.uniform(0.2, 3.0))
        rs.append(rng.normal())
    for v in range(n):
        var_lists.append([v])
        coefs.append(np.array([rng.uniform(0.3, 2.0)]))
        ss.append(rng.uniform(0.2, 2.0))
        rs.append(rng.normal())
    ptr = np.zeros(len(var_lists) + 1, np.int64)
    ptr[1:] = np.cumsum([len(v) for v in var_lists])
    return orc.FactorList(n, ptr, np.concatenate(var_lists).astype(np.int64),
                          np.concatenate(coefs).astype(float), np.array(ss), np.array(rs)).check()


@pytest.mark.parametrize("seed", range(6))
def test_tree_marginals_exact(orc, seed):
    # catches: double-counting the own message in the cavity, wrong belief sum, any error in
    # the marginal extraction; on a tree BP is exact after (diameter + 1) flooding iterations
    rng = np.random.default_rng(seed)
    fl = _random_tree_factors(orc, rng, 25 + 5 * seed)
    A = orc.dense_A(fl)
    Sigma = np.linalg.inv(A)
    mu_ex = Sigma @ orc.rhs(fl)
    mu, var, _ = orc.gabp(fl, 0.0, fl.n + 2)
    np.testing.assert_allclose(mu, mu_ex, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(var, np.diag(Sigma), rtol=1e-12, atol=1e-14)
    # damping moves the iterates, not the fixed point
    mu_d, var_d, _ = orc.gabp(fl, 0.5, 400)
    np.testing.assert_allclose(mu_d, mu_ex, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(var_d, np.diag(Sigma), rtol=1e-9, atol=1e-12)


def test_loopy_fixed_point_is_exact_mean(orc):
    # the converged loopy GaBP mean equals A^-1 b (Weiss-Freeman; Sec. 2.3 relies on it)
    p = gabp_synth.make_problem(20, 14, 0.3, 11, n_uniform=40, sigma=0.1)
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    mu_ex = orc.exact_mean(fl, p.nx)
    for beta in (0.5, 0.3):
        mu, var, _ = orc.gabp(fl, beta, 2500)
        assert np.linalg.norm(mu - mu_ex) / np.linalg.norm(mu_ex) < 1e-10
        assert orc.residual(fl, mu) < 1e-11
    # variances are only approximate on a loopy graph (Sec. 2.3): positive, same order as exact
    ex_var = orc.exact_variances(fl)
    assert np.all(var > 0)
    assert 0.05 < np.median(var / ex_var) < 20


def test_sparse_and_band_exact_solves_agree(orc):
    p = gabp_synth.make_problem(33, 21, 0.05, 2, n_tracks=3, per_track=30, sigma=0.05)
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    a = orc.exact_mean(fl, p.nx, "band")
    b = orc.exact_mean(fl, p.nx, "sparse")
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10


def test_residual_definition(orc):
    p = gabp_synth.make_problem(10, 8, 0.3, 4, n_uniform=12)
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    mu_ex = orc.exact_mean(fl, p.nx)
    assert orc.residual(fl, mu_ex) < 1e-12
    d = np.random.default_rng(0).normal(size=fl.n) * 1e-3
    A = orc.dense_A(fl)
    b = orc.rhs(fl)
    assert orc.residual(fl, mu_ex + d) == pytest.approx(np.linalg.norm(A @ d) / np.linalg.norm(b),
                                                        rel=1e-8)


def test_initialisations(orc):
    p = gabp_synth.make_problem(6, 5, 0.3, 1, n_uniform=7)
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    me, ml = orc.init_messages(fl, "cold")
    np.testing.assert_allclose(ml, np.repeat(fl.s, np.diff(fl.ptr)) * fl.coef ** 2)
    assert np.all(me == 0)
    me, ml = orc.init_messages(fl, "paper")
    assert np.all(ml == 1e-8) and np.all(me == 0)
    rng = np.random.default_rng(2)
    mu0 = rng.normal(size=fl.n)
    lam0 = rng.uniform(0.5, 3, fl.n)
    me, ml = orc.init_messages(fl, "warm", mu0, lam0)
    be, bl = orc.beliefs(fl, me, ml)
    np.testing.assert_allclose(bl, lam0, rtol=1e-14)
    np.testing.assert_allclose(be / bl, mu0, rtol=1e-13, atol=1e-14)


def test_cold_start_bounds_message_precision(orc):
    # the cold start is the upper bound s a_v^2 of every later precision message
    p = gabp_synth.make_problem(12, 9, 0.2, 3, n_uniform=20)
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    _, ml0 = orc.init_messages(fl, "cold")
    for it in (1, 5, 50):
        _, _, (me, ml) = orc.gabp(fl, 0.3, it)
        assert np.all(ml <= ml0 * (1 + 1e-14)) and np.all(ml >= 0)
