"""Pins of the oracle's prior mean (Sec. 2.2: the prior N(f_b, Sigma) has a mean f_b).

With f_b the cell factors become exp(-(gamma/2)(l_c . f - l_c . f_b)^2), so the posterior mean
solves A mu = gamma L^T L f_b + H^T R^-1 y.  Checked against what the mathematics fixes:
  * without observations the posterior is the prior, so the exact mean is f_b itself and
    converged GaBP reaches it;
  * the shift identity: mu(f_b, y) = f_b + mu(0, y - H f_b), with H written out here from the
    bilinear rule (a wrong sign or a dropped target fails it).
"""
import numpy as np
import pytest

import gabp_synth


def _H_apply(p, x):
    """H x for the bilinear rows of the observations, written out from the locations."""
    j0 = np.minimum(np.floor(p.obs_x), p.nx - 2).astype(int)
    i0 = np.minimum(np.floor(p.obs_y), p.ny - 2).astype(int)
    fu, fv = p.obs_x - j0, p.obs_y - i0
    X = x.reshape(p.ny, p.nx)
    return ((1 - fu) * (1 - fv) * X[i0, j0] + fu * (1 - fv) * X[i0, j0 + 1] + (1 - fu) * fv * X[i0 + 1, j0]
            + fu * fv * X[i0 + 1, j0 + 1])


@pytest.mark.parametrize("gamma", [1.0, 2.5])
def test_without_observations_the_mean_is_the_prior_mean(orc, gamma):
    nx, ny = 30, 24
    fb = np.random.default_rng(1).standard_normal(nx * ny)
    e = np.zeros(0)
    fl = orc.build_factors(nx, ny, 0.6, e, e, e, e, gamma, prior_mean=fb)
    np.testing.assert_allclose(orc.exact_mean(fl, nx), fb, atol=1e-11)
    mu, _, _ = orc.gabp(fl, 0.5, 800)
    np.testing.assert_allclose(mu, fb, atol=1e-10)


def test_shift_identity(orc):
    p = gabp_synth.make_problem(41, 33, 0.3, 2, n_uniform=120, n_tracks=2, per_track=40, sigma=(0.02, 0.1))
    fb = np.random.default_rng(3).standard_normal(p.n) * 2.0
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, prior_mean=fb)
    mu = orc.exact_mean(fl, p.nx)
    fl0 = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y - _H_apply(p, fb), p.noise_var)
    np.testing.assert_allclose(mu, fb + orc.exact_mean(fl0, p.nx), atol=1e-10)
    # converged GaBP with the targets reaches the same mean
    mu_g, _, _ = orc.gabp(fl, 0.5, 1000)
    assert np.linalg.norm(mu_g - mu) / np.linalg.norm(mu) < 1e-8


def test_targets_are_rows_of_L_times_the_mean(orc):
    nx, ny, kappa = 6, 5, 0.4
    fb = np.arange(nx * ny, dtype=float) ** 1.5
    pf = orc.with_prior_mean(orc.prior_factors(nx, ny, kappa), fb)
    # L written out: kappa^2 + deg on the diagonal, -1 per existing neighbour
    L = np.zeros((nx * ny, nx * ny))
    for i in range(ny):
        for j in range(nx):
            v = i * nx + j
            nb = [(i, j - 1), (i, j + 1), (i - 1, j), (i + 1, j)]
            nb = [(a, b) for a, b in nb if 0 <= a < ny and 0 <= b < nx]
            L[v, v] = kappa ** 2 + len(nb)
            for a, b in nb:
                L[v, a * nx + b] = -1.0
    np.testing.assert_allclose(pf.r, L @ fb, rtol=1e-12, atol=1e-11)

