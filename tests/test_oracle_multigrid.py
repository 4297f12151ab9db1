"""Pins of the oracle's multigrid warm start (oracle/multigrid.py) to what the SPDE and the
procedure fix: the coarse levels discretise the same field, upscaling copies parents, and
a multigrid start reaches the exact posterior with fewer fine iterations."""
import numpy as np
import pytest

import gabp_synth
import oracle
from oracle import multigrid as mg


def _prior_column(n, kappa, gamma):
    fl = oracle.prior_factors(n, n, kappa, gamma)
    A = oracle.dense_A(fl)
    c = (n // 2) * n + n // 2
    e = np.zeros(n * n)
    e[c] = 1.0
    return np.linalg.solve(A, e), c


def test_levels_keep_the_prior_variance():
    # kappa_k = 2^k kappa, gamma_k = gamma / 4^k discretise the same Matern field: the marginal
    # prior variance at an interior node stays near the continuum value 1 / (4 pi kappa^2 gamma)
    kappa, gamma, n0 = 0.2, 1.0, 64
    cont = 1.0 / (4 * np.pi * kappa ** 2 * gamma)
    v = []
    for k in range(3):
        nk, _, kk, gk, _, _ = mg.level_problem(n0, n0, kappa, gamma, [], [], k)
        col, c = _prior_column(nk, kk, gk)
        v.append(col[c])
    assert abs(v[0] / cont - 1) < 0.05
    for k in (1, 2):
        assert abs(v[k] / v[0] - 1) < 0.15, v   # an unscaled gamma would give 0.26, 0.07


def test_levels_keep_the_prior_correlation_length():
    # correlation between the centre and a node 8 target cells away: the same physical distance
    # at every level (8, 4, 2 cells), close to the Matern value r K1(r) at r = 8 kappa
    from scipy.special import k1
    kappa, n0 = 0.2, 64
    rho = []
    for k in range(3):
        nk, _, kk, gk, _, _ = mg.level_problem(n0, n0, kappa, 1.0, [], [], k)
        col, c = _prior_column(nk, kk, gk)
        rho.append(col[c + 8 // (1 << k)] / col[c])
    r = 8 * kappa
    assert abs(rho[0] - r * k1(r)) < 0.02
    for k in (1, 2):
        assert abs(rho[k] - rho[0]) < 0.05, rho   # an unscaled kappa would give 0.69, 0.93


def test_level_shapes_and_observation_coordinates():
    assert mg.level_shape(64, 48, 1) == (32, 24)
    assert mg.level_shape(67, 45, 1) == (34, 23)
    assert mg.level_shape(67, 45, 3) == (9, 6)
    nx, ny, kk, gk, ox, oy = mg.level_problem(67, 45, 0.1, 2.0, [0.0, 66.0, 13.5], [44.0, 0.5, 7.0], 1)
    assert (nx, ny) == (34, 23) and kk == pytest.approx(0.2) and gk == pytest.approx(0.5)
    np.testing.assert_allclose(ox, [0.0, 33.0, 6.75])
    np.testing.assert_allclose(oy, [22.0, 0.25, 3.5])
    # a location past the level's last node is clamped onto it
    _, _, _, _, ox2, _ = mg.level_problem(67, 45, 0.1, 1.0, [66.0], [0.0], 3)
    assert ox2[0] == 8.0


def test_upscale_copies_parents():
    mu_c = np.arange(6, dtype=float)            # 2 rows x 3 columns
    var_c = 1.0 / (10.0 + np.arange(6))
    mu, lam = mg.upscale(mu_c, var_c, 3, 2, 5, 4)   # target 4 rows x 5 columns
    mu = mu.reshape(4, 5)
    lam = lam.reshape(4, 5)
    expect = np.array([[0, 0, 1, 1, 2], [0, 0, 1, 1, 2], [3, 3, 4, 4, 5], [3, 3, 4, 4, 5]], float)
    np.testing.assert_array_equal(mu, expect)
    np.testing.assert_allclose(lam, 10.0 + expect)


def test_solve_level_retries_a_diverging_level_with_more_damping():
    p = gabp_synth.make_problem(64, 64, 0.05, 4, n_uniform=40, n_tracks=0, per_track=0, sigma=(0.05, 0.05))
    nxk, nyk, kk, gk, ox, oy = mg.level_problem(p.nx, p.ny, p.kappa, 1.0, p.obs_x, p.obs_y, 3)
    fl = oracle.build_factors(nxk, nyk, kk, ox, oy, p.y, p.noise_var, gamma=gk)
    m, _, _ = oracle.gabp(fl, 0.3, 300)
    assert not oracle.residual(fl, m) < 1.0          # diverges at 0.3
    _, _, r, b, ok = mg.solve_level(fl, 0.3, 300)
    assert ok and b == pytest.approx(0.65) and r < 1e-6


def test_multigrid_start_converges_to_the_exact_mean_in_fewer_iterations():
    # sparse observations and a long correlation length: the regime where the paper uses
    # multigrid.  Same fixed point (the start does not change it), fewer fine iterations.
    p = gabp_synth.make_problem(64, 64, 0.05, 4, n_uniform=40, n_tracks=0, per_track=0, sigma=(0.05, 0.05))
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    exact = oracle.exact_mean(fl, p.nx)
    mu0, lam0, info = mg.multigrid_init(p.nx, p.ny, p.kappa, 1.0, p.obs_x, p.obs_y, p.y, p.noise_var,
                                        levels=4, beta=0.3, iters=300)
    # 40 observations on the 8 x 8 coarsest level: GaBP diverges at damping 0.3 there and the
    # level is re-run with damping 0.65; the finer levels converge at 0.3
    assert info[3][1] == pytest.approx(0.65) and info[3][2]
    assert info[2][1] == pytest.approx(0.3) and info[1][1] == pytest.approx(0.3)
    assert all(r < 1e-4 for r, _, _ in info.values())

    def iters_to(tol, **init):
        mu, _, msg = oracle.gabp(fl, 0.3, 0, **init)
        for it in range(0, 4000, 20):
            if oracle.residual(fl, mu) <= tol:
                return it, mu
            mu, _, msg = oracle.gabp(fl, 0.3, 20, messages=msg)
        return None, mu

    it_cold, _ = iters_to(1e-6, init="cold")
    it_mg, mu_mg = iters_to(1e-6, init="warm", mu0=mu0, lam0=lam0)
    assert it_cold is not None and it_mg is not None
    assert it_mg < 0.7 * it_cold, (it_mg, it_cold)
    # the fixed point is the exact posterior mean whatever the start (slow tail at kappa 0.05)
    mu_fin, _, _ = oracle.gabp(fl, 0.3, 3000, init="warm", mu0=mu0, lam0=lam0)
    assert np.linalg.norm(mu_fin - exact) / np.linalg.norm(exact) < 1e-4
