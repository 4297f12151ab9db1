"""The alpha = 4 prior (cell factors = rows of L^2, 13 slots) on the GPU against the oracle's
(oracle.prior_factors(..., alpha=4)): iterates, marginals, residual, convergence to the exact
mean, the message-change quantity, and the entry points that need alpha = 2."""
import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built, rel_l2, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _fl(orc, p):
    return orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, alpha=4)


def _problem(nx, ny, seed=3):
    return gabp_synth.make_problem(nx, ny, 0.3, seed, n_uniform=max(4, nx * ny // 10), n_tracks=1,
                                   per_track=nx, sigma=(0.05, 0.15))


@pytest.mark.parametrize("shape", [(23, 17), (5, 4), (64, 3), (40, 37)])
def test_fp64_iterates_match_oracle(orc, shape):
    p = _problem(*shape)
    fl = _fl(orc, p)
    mu0, var0, _ = orc.gabp(fl, 0.5, 60)
    with solver(p, "fp64", alpha=4) as s:
        s.iterate(60, 0.5)
        mu, var = s.marginals()
        res = s.residual()
        st = s.stats()
    assert rel_l2(mu, mu0) < 1e-10
    assert np.max(np.abs(var - var0) / var0) < 1e-10
    assert res == pytest.approx(orc.residual(fl, mu0), rel=1e-8)
    # slots: 13 per interior cell, fewer at the border (the oracle's factor sizes)
    assert st["edges"] == fl.ne and st["kernel"] == 2


def test_fp32_iterates_match_oracle(orc):
    p = _problem(96, 80, seed=5)
    fl = _fl(orc, p)
    mu0, var0, _ = orc.gabp(fl, 0.5, 80)
    with solver(p, "fp32", alpha=4) as s:
        s.iterate(80, 0.5)
        mu, var = s.marginals()
    assert rel_l2(mu, mu0) < 1e-4
    assert np.max(np.abs(var - var0) / var0) < 1e-4


@pytest.mark.parametrize("prec,tol,err", [("fp64", 1e-9, 1e-6), ("fp32", 1e-5, None)])
def test_converges_to_the_exact_mean(orc, prec, tol, err):
    """Iterated to a relative residual (FP32 messages reach 1e-5; their rounding floor for this
    prior is near 2e-6), confirmed by the oracle; FP64 also against the exact mean."""
    p = _problem(48, 40, seed=7)
    fl = _fl(orc, p)
    with solver(p, prec, alpha=4, tol=tol, check_every=20, max_iters=40000) as s:
        s.iterate(-1, 0.5)
        mu, _ = s.marginals(want_var=False)
        res = s.residual()
    assert res <= tol
    assert orc.residual(fl, mu) == pytest.approx(res, rel=1e-3)
    if err is not None:
        assert rel_l2(mu, orc.exact_mean(fl, p.nx)) < err


def _fp32_values(buf):
    # messages as FP32 values (np.array_equal treats -0 and +0 as equal)
    return buf.view(np.float32)


@pytest.mark.parametrize("shape", [(23, 17), (5, 4), (2, 9), (64, 3), (40, 37), (120, 61), (173, 90), (610, 404)])
@pytest.mark.parametrize("ty,run", [(8, 0), (4, 0), (8, 3)])
def test_fused_kernel_matches_split(shape, ty, run):
    """The fused alpha = 4 tile kernel gives the split kernels' messages bit for bit: shapes
    smaller than a tile, with ragged edge tiles in both directions, with interior tiles (a
    window whose every source cell exists), and large enough for long runs of tiles down each
    column; both tile heights (28 x 8: one cell per thread; 28 x 4: one warp per row); runs of
    3 and the chosen length (carried belief rows)."""
    from paper_2404_12968_gb300 import GABP_KERNEL_FUSED, GABP_KERNEL_SPLIT
    p = _problem(*shape, seed=11)
    out = []
    for kern, extra in ((GABP_KERNEL_SPLIT, {}), (GABP_KERNEL_FUSED, {"tile_x": 28, "tile_y": ty, "tile_run": run})):
        with solver(p, "fp32", alpha=4, kernel=kern, **extra) as s:
            s.iterate(25, 0.5)
            st = s.stats()
            out.append(_fp32_values(s.get_messages()))
        assert st["kernel"] == kern
        if kern == GABP_KERNEL_FUSED:
            assert st["tile_y"] == ty and (run == 0 or st["tile_run"] == run) and st["tile_run"] >= 1
    assert np.array_equal(out[0], out[1])


def test_fused_kernel_is_the_fp32_default():
    from paper_2404_12968_gb300 import GABP_KERNEL_FUSED
    p = _problem(60, 44)
    with solver(p, "fp32", alpha=4) as s:
        assert s.stats()["kernel"] == GABP_KERNEL_FUSED and s.stats()["tile_y"] == 8
    with solver(p, "fp64", alpha=4) as s:
        assert s.stats()["kernel"] == 2


def test_message_change_and_checkpoint(orc):
    from oracle import early_stop as es
    p = _problem(30, 26, seed=9)
    fl = _fl(orc, p)
    _, _, m1 = orc.gabp(fl, 0.5, 9)
    _, _, m2 = orc.gabp(fl, 0.5, 1, messages=m1)
    with solver(p, "fp64", alpha=4) as s:
        s.iterate(10, 0.5)
        assert s.message_change() == pytest.approx(es.message_change(m2, m1), rel=1e-10)
        ck = s.get_messages()
        assert ck.nbytes == (2 * 13 * p.n + 8 * p.m) * 8
        s.iterate(7, 0.5)
        a = s.get_messages()
        s.set_messages(ck)
        s.iterate(7, 0.5)
        assert np.array_equal(s.get_messages(), a)


def test_alpha4_argument_and_state_errors():
    from paper_2404_12968_gb300 import (GABP_KERNEL_FUSED, GABP_KERNEL_SPLIT, GABP_KERNEL_TMA, GabpError, Multigrid,
                                        Pairwise)
    p = _problem(24, 20)
    with pytest.raises(GabpError, match="alpha must be 2 or 4"):
        solver(p, "fp32", alpha=3)
    with pytest.raises(GabpError, match="fused or the split kernels"):
        solver(p, "fp32", alpha=4, kernel=GABP_KERNEL_TMA)
    with pytest.raises(GabpError, match="needs FP32"):
        solver(p, "fp64", alpha=4, kernel=GABP_KERNEL_FUSED)
    with pytest.raises(GabpError, match="tile shape"):
        solver(p, "fp32", alpha=4, tile_x=28, tile_y=16)
    with pytest.raises(GabpError, match="tile shape"):
        solver(p, "fp32", alpha=4, kernel=GABP_KERNEL_SPLIT, tile_x=28, tile_y=8)
    with solver(p, "fp32", alpha=4) as s:
        with pytest.raises(GabpError, match="alpha = 4"):
            s.warm_start(np.zeros(p.n), np.ones(p.n))
        with pytest.raises(GabpError, match="alpha = 4"):
            Multigrid(s, 2)
        with pytest.raises(GabpError, match="alpha = 2"):
            Pairwise(s)
