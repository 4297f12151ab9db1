"""Prior mean (Sec. 2.2: the prior N(f_b, Sigma)) on the GPU, against the oracle.

The cell factors get the targets r_c = (L f_b)_c.
* FP64 iterates with a prior mean equal the oracle's GaBP iterates with the same targets
  (1e-10), for the fused and split kernels, and the residual includes the prior term;
* every FP32 kernel gives the same bits with a prior mean; FP32 tracks the oracle;
* the converged mean without observations is f_b itself; clearing the mean restores the
  original problem; contexts with a prior mean refuse multigrid and the pairwise form.
"""
import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built, oracle_factors, rel_l2, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("kernel", [1, 2])   # fused, split
def test_fp64_iterates_with_prior_mean_match_oracle(orc, kernel):
    p = gabp_synth.make_problem(57, 43, 0.2, 4, n_uniform=250, n_tracks=2, per_track=60, sigma=(0.02, 0.1))
    fb = np.random.default_rng(7).standard_normal(p.n) * 1.5
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, prior_mean=fb)
    mu_o, var_o, _ = orc.gabp(fl, 0.5, 90)
    with solver(p, "fp64", kernel=kernel) as s:
        s.set_prior_mean(fb)
        s.iterate(90, 0.5)
        mu, var = s.marginals()
        res = s.residual()
    assert rel_l2(mu, mu_o) < 1e-10
    assert np.max(np.abs(var - var_o) / var_o) < 1e-10
    assert res == pytest.approx(orc.residual(fl, mu), rel=1e-8)


@pytest.mark.parametrize("shape", [(68, 45), (256, 130), (61, 30)])
def test_fp32_kernels_bit_identical_with_prior_mean(shape):
    nx, ny = shape
    p = gabp_synth.make_problem(nx, ny, 0.05, 9, n_tracks=4, per_track=nx, n_uniform=nx * ny // 20, sigma=(0.02, 0.1))
    fb = np.sin(np.arange(p.n) * 0.01) * 3.0
    variants = [(2, (0, 0)), (1, (32, 8)), (1, (64, 16)), (4, (30, 32))]
    if nx % 4 == 0:
        variants += [(3, (30, 14)), (3, (30, 22))]
    bufs = []
    for kernel, tile in variants:
        with solver(p, "fp32", kernel=kernel, tile_x=tile[0], tile_y=tile[1]) as s:
            s.set_prior_mean(fb)
            s.iterate(41, 0.3)
            bufs.append(s.get_messages())
    for b in bufs[1:]:
        assert np.array_equal(b, bufs[0])


def test_fp32_prior_mean_tracks_oracle(orc):
    p = gabp_synth.config_small(1)
    fb = np.cos(np.arange(p.n) * 0.05) * 0.5
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, prior_mean=fb)
    mu_o, _, _ = orc.gabp(fl, 0.5, 200)
    with solver(p, "fp32") as s:
        s.set_prior_mean(fb)
        s.iterate(200, 0.5)
        mu, _ = s.marginals(want_var=False)
    assert rel_l2(mu, mu_o) < 1e-5


def test_prior_mean_alone_and_cleared(orc):
    """Without observations the converged mean is f_b (FP64); clearing the prior mean gives back
    the iterates of the original problem."""
    p = gabp_synth.make_problem(40, 32, 0.6, 3, n_uniform=0)
    fb = np.random.default_rng(5).standard_normal(p.n)
    with solver(p, "fp64") as s:
        s.set_prior_mean(fb)
        s.iterate(800, 0.5)
        mu, _ = s.marginals(want_var=False)
        assert np.max(np.abs(mu - fb)) < 1e-10
        assert s.residual() < 1e-12
    q = gabp_synth.make_problem(40, 32, 0.3, 3, n_uniform=150, sigma=0.1)
    with solver(q, "fp64") as s:
        s.iterate(50, 0.5)
        ref, _ = s.marginals(want_var=False)
        s.set_prior_mean(np.ones(q.n))
        s.set_prior_mean(None)
        s.reset()
        s.iterate(50, 0.5)
        again, _ = s.marginals(want_var=False)
    np.testing.assert_array_equal(again, ref)


def test_prior_mean_refusals():
    from paper_2404_12968_gb300 import GabpError, Multigrid, Pairwise
    p = gabp_synth.make_problem(40, 30, 0.2, 1, n_uniform=60)
    with solver(p, "fp32") as s:
        s.set_prior_mean(np.ones(p.n))
        with pytest.raises(GabpError, match="STATE"):
            Multigrid(s, 2)
        with pytest.raises(GabpError, match="STATE"):
            Pairwise(s)
        s.set_prior_mean(None)
        Pairwise(s).close()
    with solver(p, "fp32", alpha=4) as s:
        with pytest.raises(GabpError, match="STATE"):
            s.set_prior_mean(np.ones(p.n))
