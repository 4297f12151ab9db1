"""Pins of the oracle's exact solves for large grids (``oracle/exact.py``).

The preconditioned conjugate gradient solve and the banded selected inversion are checked
against things other than themselves:
  * the banded Cholesky solve (a different algorithm and code path) on ragged grids;
  * a closed form: with a single observation of row h, the posterior mean is
    C h y / (sigma^2 + h^T C h) with C = (gamma L^T L)^-1, whose columns come from the 2-D
    DCT-II diagonalisation of the zero-Neumann L (no assembly, no iteration);
  * the dense inverse (LAPACK) for diag(A^-1), and for the prior alone the DCT closed form
    diag(C)_i = sum_kl phi_kl(i)^2 / (gamma lambda_kl^2);
  * the symmetry of the multigrid preconditioner, which conjugate gradients relies on.
"""
import numpy as np
import pytest

import gabp_synth


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ex(orc):
    from oracle import exact
    return exact


@pytest.mark.parametrize("shape,kappa,seed", [((97, 61), 0.05, 1), ((128, 128), 0.02, 2), ((33, 70), 0.3, 3)])
def test_pcg_matches_band_solve(orc, ex, shape, kappa, seed):
    nx, ny = shape
    p = gabp_synth.make_problem(nx, ny, kappa, seed, n_tracks=5, per_track=nx, n_uniform=nx * ny // 40,
                                sigma=(0.02, 0.1))
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    x_band = orc.exact_mean(fl, p.nx)
    x, info = ex.exact_mean_pcg(fl, p.nx, p.ny, tol=1e-14)
    assert info["rel_residual"] <= 2e-14
    assert _rel(x, x_band) < 1e-11


def test_pcg_dct_preconditioner_matches_band_solve(orc, ex):
    p = gabp_synth.make_problem(48, 40, 0.3, 4, n_uniform=120, sigma=0.1)
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, 1.7)
    x_band = orc.exact_mean(fl, p.nx)
    x, info = ex.exact_mean_pcg(fl, p.nx, p.ny, tol=1e-14, precond="dct", kappa=p.kappa, gamma=1.7)
    assert _rel(x, x_band) < 1e-11
    # without observations the DCT preconditioner is the exact inverse of A
    q = gabp_synth.make_problem(48, 40, 0.3, 4, n_uniform=0)
    flq = orc.build_factors(q.nx, q.ny, q.kappa, q.obs_x, q.obs_y, q.y, q.noise_var)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(q.n)
    np.testing.assert_allclose(orc.apply_A(flq, ex.dct_prior_solve(v, q.nx, q.ny, q.kappa)), v, atol=1e-9)


@pytest.mark.parametrize("gamma", [1.0, 3.5])
def test_single_observation_closed_form(orc, ex, gamma):
    """One observation at a continuous location: mean = C h y / (sigma^2 + h^T C h)."""
    nx, ny, kappa = 150, 110, 0.04
    u, v, yv, s2 = 73.3, 41.8, 1.25, 0.01
    fl = orc.build_factors(nx, ny, kappa, np.array([u]), np.array([v]), np.array([yv]), np.array([s2]), gamma)
    x, _ = ex.exact_mean_pcg(fl, nx, ny, tol=1e-14)
    # bilinear row h written out here from the location (not from the oracle's weights)
    j0, i0 = int(np.floor(u)), int(np.floor(v))
    fu, fv = u - j0, v - i0
    corners = [(i0, j0, (1 - fu) * (1 - fv)), (i0, j0 + 1, fu * (1 - fv)), (i0 + 1, j0, (1 - fu) * fv),
               (i0 + 1, j0 + 1, fu * fv)]
    Ch = np.zeros(nx * ny)
    hCh = 0.0
    cols = {}
    for (i, j, w) in corners:
        cols[(i, j)] = ex.prior_covariance_column(i * nx + j, nx, ny, kappa, gamma)
        Ch += w * cols[(i, j)]
    for (i, j, w) in corners:
        hCh += w * Ch[i * nx + j]
    expect = Ch * yv / (s2 + hCh)
    # the solve stops at ||b - A x|| / ||b|| = 1e-14 and A's condition number here is about
    # 1e7 (kappa^4 = 2.6e-6 at the bottom of the prior's spectrum), so the error it leaves is
    # below 1e-7; a dropped term, a wrong weight or sign gives errors of order 1
    assert _rel(x, expect) < 1e-8
    # the prior covariance column itself: L^T L C e_k = e_k / gamma
    e = np.zeros(nx * ny)
    e[i0 * nx + j0] = 1.0
    q = orc.build_factors(nx, ny, kappa, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), gamma)
    np.testing.assert_allclose(orc.apply_A(q, cols[(i0, j0)]), e, atol=1e-9)


def test_pcg_without_observations_is_zero(orc, ex):
    fl = orc.build_factors(40, 30, 0.1, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    x, info = ex.exact_mean_pcg(fl, 40, 30)
    assert np.all(x == 0.0) and info["iterations"] == 0


def test_multigrid_preconditioner_is_symmetric(orc, ex):
    from oracle.exact import _vcycle
    p = gabp_synth.make_problem(131, 77, 0.05, 5, n_tracks=4, per_track=150, n_uniform=300, sigma=(0.02, 0.1))
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    A = ex.assemble_csr(fl)
    levels, Ps, lu = ex.mg_hierarchy(A, p.nx, p.ny, coarsest=16)
    assert len(levels) >= 3
    rng = np.random.default_rng(3)
    u, w = rng.standard_normal(p.n), rng.standard_normal(p.n)
    Mu, Mw = _vcycle(levels, Ps, lu, 0, u, 2), _vcycle(levels, Ps, lu, 0, w, 2)
    assert abs(Mu @ w - u @ Mw) < 1e-10 * abs(Mu @ w)
    assert Mu @ u > 0 and Mw @ w > 0
    # the assembled matrix is the factor list's A
    np.testing.assert_allclose(A @ u, orc.apply_A(fl, u), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("alpha", [2, 4])
def test_selected_inversion_matches_dense_inverse(orc, ex, alpha):
    p = gabp_synth.make_problem(30, 26, 0.2, 6, n_tracks=3, per_track=30, n_uniform=40, sigma=(0.02, 0.1))
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, 1.0, alpha)
    v = ex.exact_variances_band(fl, p.nx)
    dense = np.diag(np.linalg.inv(orc.dense_A(fl)))
    np.testing.assert_allclose(v, dense, rtol=1e-10)


def test_selected_inversion_prior_closed_form(orc, ex):
    """Prior alone: diag((gamma L^2)^-1)_i = sum_kl phi_k(x_i)^2 phi_l(y_i)^2 / (gamma lambda_kl^2),
    with the orthonormal 1-D DCT-II basis phi written out here."""
    nx, ny, kappa, gamma = 40, 32, 0.15, 2.0
    fl = orc.build_factors(nx, ny, kappa, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), gamma)
    v = ex.exact_variances_band(fl, nx)

    def basis(N):
        k = np.arange(N)[:, None]
        i = np.arange(N)[None, :]
        phi = np.cos(np.pi * k * (2 * i + 1) / (2 * N)) * np.sqrt(2.0 / N)
        phi[0] /= np.sqrt(2.0)
        return phi                     # phi[k, i]

    px, py = basis(nx), basis(ny)
    lam = gabp_synth.neumann_eigenvalues(nx, ny, kappa)          # (ny, nx): [l, k]
    expect = (py ** 2).T @ (1.0 / (gamma * lam ** 2)) @ (px ** 2)   # [i_y, i_x]
    np.testing.assert_allclose(v, expect.reshape(-1), rtol=1e-10)


def test_selected_inversion_refuses_oversized_band(orc, ex):
    fl = orc.build_factors(4096, 64, 0.1, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    with pytest.raises(ValueError):
        ex.exact_variances_band(fl, 4096)
