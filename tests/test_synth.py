"""The paper's synthetic setting (gabp_synth.paper_synthetic): the unit-spacing rescaling of the
prior keeps the marginal variance the paper fixes with q (App. E and the white-noise scaling)."""
import math

import numpy as np
import pytest
from scipy import fft as sfft

import gabp_synth


def _centre_variance(p):
    # Var(f_c) = e_c^T (gamma L^T L)^-1 e_c = ||L^-1 e_c||^2 / gamma (L symmetric), by a spectral solve
    n = p.nx
    e = np.zeros((n, n))
    e[n // 2, n // 2] = 1.0
    lam = gabp_synth.neumann_eigenvalues(n, n, p.kappa)
    v = sfft.idctn(sfft.dctn(e, type=2, norm="ortho") / lam, type=2, norm="ortho")
    return float(np.sum(v * v)) / p.gamma


def test_marginal_variance_is_sigma_squared():
    # sigma = 1.1: the interior marginal variance of the discretised prior is sigma^2 up to the
    # finite-difference error, at every grid size (kappa h and gamma scale together)
    for side in (64, 128, 256):
        p = gabp_synth.paper_synthetic(side, 0.05, 0)
        assert abs(_centre_variance(p) / 1.21 - 1.0) < 0.1, side


def test_rescaled_parameters_and_observations():
    p = gabp_synth.paper_synthetic(256, 0.05, 1)
    kappa = math.sqrt(2.0) / 0.15
    assert p.kappa == pytest.approx(kappa / 256)
    assert p.gamma == pytest.approx(256 ** 2 / (1.21 * 4 * math.pi * kappa ** 2))
    assert p.m == round(0.05 * 256 * 256)
    # grid-point observations, distinct, values = truth + noise of std 0.01
    assert np.all(p.obs_x == np.round(p.obs_x)) and np.all(p.obs_y == np.round(p.obs_y))
    idx = (p.obs_y * 256 + p.obs_x).astype(int)
    assert np.unique(idx).size == p.m
    resid = p.y - p.truth.reshape(-1)[idx]
    assert abs(resid.std() - 0.01) < 0.001 and np.allclose(p.noise_var, 1e-4, rtol=1e-12)


def test_exact_posterior_rmse_matches_the_papers_inla_column():
    """The exact posterior mean's RMSE against the truth on the paper's synthetic setting at
    256^2 (5 % and 10 % observed, mean of three ground truths) is the paper's R-INLA RMSE
    (golden table, Sec. 4.1) within 10 %: the generator's prior (unit square, h = 1/N,
    lengthscale 0.15, sigma 1.1) and noise (0.01) reproduce the paper's data."""
    import os
    import oracle
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(__file__), "golden", "table1_rmse.txt"))
            if ln.strip() and not ln.startswith("#")]
    inla = {(int(r[0]), float(r[1])): float(r[2]) for r in rows}
    for frac in (0.05, 0.10):
        rmse = []
        for seed in range(3):
            p = gabp_synth.paper_synthetic(256, frac, seed)
            fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, gamma=p.gamma)
            mu = oracle.exact_mean(fl, p.nx, method="sparse")
            rmse.append(np.sqrt(np.mean((mu - p.truth.reshape(-1)) ** 2)))
        assert abs(np.mean(rmse) / inla[(256, frac)] - 1.0) < 0.10, (frac, np.mean(rmse))
