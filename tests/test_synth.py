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
    # grid-point observations, distinct, values = truth + noise of std 0.1
    assert np.all(p.obs_x == np.round(p.obs_x)) and np.all(p.obs_y == np.round(p.obs_y))
    idx = (p.obs_y * 256 + p.obs_x).astype(int)
    assert np.unique(idx).size == p.m
    resid = p.y - p.truth.reshape(-1)[idx]
    assert abs(resid.std() - 0.1) < 0.01 and np.allclose(p.noise_var, 0.01, rtol=1e-15)
