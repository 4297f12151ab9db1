"""Pins of the oracle's alpha = 4 prior (rows of L^2 as cell factors; Sec. 3.1 with alpha/2 = 2,
App. C powers of the operator) to what the SPDE fixes: the assembled precision's spectrum, the
Matern (nu = 3) marginal variance and correlation, and the exact posterior mean at convergence."""
import math

import numpy as np
import pytest

import gabp_synth
import oracle


def _neumann_eigs(nx, ny, kappa):
    # eigenvalues of kappa^2 I + graph Laplacian with zero-Neumann ends (cosine basis)
    kx = 4.0 * np.sin(np.pi * np.arange(nx) / (2.0 * nx)) ** 2
    ky = 4.0 * np.sin(np.pi * np.arange(ny) / (2.0 * ny)) ** 2
    return (kappa * kappa + ky[:, None] + kx[None, :]).reshape(-1)


def test_precision_spectrum_is_gamma_lambda_to_the_fourth():
    # P = gamma (L^2)^T L^2 = gamma L^4: eigenvalues gamma * lambda^4 of the Neumann operator;
    # a wrong coefficient, boundary row or slot would move them
    nx, ny, kappa, gamma = 9, 7, 0.4, 1.7
    fl = oracle.prior_factors(nx, ny, kappa, gamma, alpha=4)
    ev = np.sort(np.linalg.eigvalsh(oracle.dense_A(fl)))
    expect = np.sort(gamma * _neumann_eigs(nx, ny, kappa) ** 4)
    # eigenvalue accuracy is relative to the largest one
    np.testing.assert_allclose(ev, expect, rtol=1e-10, atol=1e-13 * expect.max())


def _prior_cov_column(n, kappa, gamma=1.0):
    fl = oracle.prior_factors(n, n, kappa, gamma, alpha=4)
    A = oracle.dense_A(fl)
    c = (n // 2) * n + n // 2
    e = np.zeros(n * n)
    e[c] = 1.0
    return np.linalg.solve(A, e), c


def test_marginal_variance_is_the_matern_nu3_value():
    # (kappa^2 - Delta)^2 f = W in 2-D: Matern with nu = alpha - d/2 = 3, variance
    # Gamma(nu) / (Gamma(nu + 1) 4 pi kappa^(2 nu)) = 1 / (12 pi kappa^6) per unit gamma
    kappa, gamma = 0.35, 2.0
    col, c = _prior_cov_column(48, kappa, gamma)
    cont = 1.0 / (12.0 * math.pi * kappa ** 6 * gamma)
    assert abs(col[c] / cont - 1.0) < 0.08, (col[c], cont)


def test_correlation_is_the_matern_nu3_value():
    # rho(r) = (kappa r)^3 K_3(kappa r) / (2^2 Gamma(3)) at r = 4, 8 cells
    from scipy.special import kv
    kappa = 0.35
    col, c = _prior_cov_column(48, kappa)
    for r in (4, 8):
        rho = col[c + r] / col[c]
        x = kappa * r
        assert abs(rho - x ** 3 * kv(3, x) / 8.0) < 0.03, (r, rho)


def test_interior_row_and_bandwidth():
    fl = oracle.prior_factors(11, 10, 0.3, 1.0, alpha=4)
    c = 5 * 11 + 5
    sl = slice(fl.ptr[c], fl.ptr[c + 1])
    assert fl.ptr[c + 1] - fl.ptr[c] == 13
    # (kappa^2 + 4)^2 + 4 at the centre, -2 (kappa^2 + 4) at the four neighbours, 2 on the
    # diagonals and 1 two steps away: the two-step paths of L
    a = 0.09 + 4.0
    np.testing.assert_allclose(fl.coef[sl], [a * a + 4] + [-2 * a] * 4 + [2.0] * 4 + [1.0] * 4, rtol=1e-14)
    assert oracle.half_bandwidth(fl) == 4 * 11
    assert oracle.half_bandwidth(oracle.prior_factors(11, 10, 0.3)) == 2 * 11


def test_converged_gabp_mean_is_the_exact_mean():
    p = gabp_synth.make_problem(20, 17, 0.3, 2, n_uniform=80, n_tracks=1, per_track=20, sigma=0.1)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, alpha=4)
    exact = oracle.exact_mean(fl, p.nx)
    # the banded solve with the alpha = 4 bandwidth is exact: dense check
    np.testing.assert_allclose(oracle.dense_A(fl) @ exact, oracle.rhs(fl), rtol=1e-9, atol=1e-9)
    mu, var, _ = oracle.gabp(fl, 0.5, 3000)
    assert np.all(np.isfinite(mu)) and np.all(var > 0)
    assert np.linalg.norm(mu - exact) / np.linalg.norm(exact) < 1e-8
    assert oracle.residual(fl, mu) < 1e-8
