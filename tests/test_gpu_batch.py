"""Batched GaBP (one persistent launch per iteration over many problems of uneven sizes)
against single-problem contexts and the CPU oracle."""
import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built, oracle_factors, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _mixed_batch():
    """Uneven sizes: every width class of the TMA kernel's copies, a problem smaller than one
    tile, one without observations, ragged tile edges."""
    probs = gabp_synth.config_batch(seed=3, count=6, lo=48, hi=200)
    probs += [gabp_synth.make_problem(64, 37, 0.1, 1, n_uniform=200, n_tracks=2, per_track=64, sigma=(0.02, 0.1)),
              gabp_synth.make_problem(61, 30, 0.1, 2, n_uniform=150, sigma=0.05),
              gabp_synth.make_problem(7, 5, 0.2, 3, n_uniform=6, sigma=0.1),
              gabp_synth.make_problem(33, 62, 0.05, 4),
              gabp_synth.make_problem(120, 91, 0.03, 5, n_tracks=3, per_track=200, sigma=0.05),
              gabp_synth.make_problem(62, 31, 0.08, 6, n_uniform=120, n_tracks=2, per_track=60, sigma=0.05)]
    # widths: multiples of 4 (tensor copies), 2 mod 4 (planes by tensor copies, index by
    # cp.async) and odd (cp.async)
    assert {p.nx % 4 for p in probs} >= {0, 1, 2} and any(p.nx % 2 for p in probs)
    return probs


@pytest.mark.parametrize("kernel,tile_y", [("sweep", 32), ("tma", 14), ("tma", 22), ("tma", 30)])
def test_batch_lockstep_bit_identical_to_single_contexts(kernel, tile_y):
    from paper_2404_12968_gb300 import Batch, GABP_KERNEL_SWEEP, GABP_KERNEL_TMA
    probs = _mixed_batch()
    k = GABP_KERNEL_TMA if kernel == "tma" else GABP_KERNEL_SWEEP
    with Batch(probs, kernel=k, tile_y=tile_y) as b:
        assert b.strip_height == tile_y and b.kernel == k
        b.iterate(37, 0.3)
        means = [b.marginals(i)[0] for i in range(len(probs))]
        for i, p in enumerate(probs):
            with solver(p, "fp32", kernel=GABP_KERNEL_SWEEP, tile_x=30, tile_y=32) as s:
                s.iterate(37, 0.3)
                mu, _ = s.marginals(want_var=False)
            assert np.array_equal(mu, means[i]), i
            assert b.stats(i)["iterations"] == 37


@pytest.mark.parametrize("kernel", ["sweep", "tma"])
def test_batch_until_tolerance_matches_oracle_residual(orc, kernel):
    """Problems leave the active set as they converge (the TMA kernel's compacted work list,
    the sweep kernel's flags); the oracle confirms every final residual."""
    from paper_2404_12968_gb300 import Batch, GABP_KERNEL_SWEEP, GABP_KERNEL_TMA
    probs = gabp_synth.config_batch(seed=4, count=10, lo=64, hi=256)
    k = GABP_KERNEL_TMA if kernel == "tma" else GABP_KERNEL_SWEEP
    with Batch(probs, tol=1e-5, check_every=20, kernel=k) as b:
        assert b.kernel == k
        b.iterate(-1, 0.3)
        res = b.residuals()
        assert np.all(res <= 1e-5)
        its = [b.stats(i)["iterations"] for i in range(len(probs))]
        assert len(set(its)) > 1   # problems converge (and stop) at different counts
        for i, p in enumerate(probs):
            mu, _ = b.marginals(i)
            fl = oracle_factors(orc, p)
            assert orc.residual(fl, mu) == pytest.approx(res[i], rel=1e-3)


def test_batch_64_instances_config(orc):
    """The 64-instance configuration: sides log-uniform in [128, 1024], kappa ~ U[0.02, 0.2],
    4-32 tracks; every problem to relative residual 1e-5, checked by the oracle."""
    from paper_2404_12968_gb300 import Batch, GABP_KERNEL_SWEEP, GABP_KERNEL_TMA
    probs = gabp_synth.config_batch(seed=0)
    assert len(probs) == 64
    with Batch(probs, tol=1e-5) as b:   # the autotuner's choice
        assert (b.kernel, b.strip_height) in [(GABP_KERNEL_SWEEP, h) for h in (16, 32, 64, 128)] + \
            [(GABP_KERNEL_TMA, 14), (GABP_KERNEL_TMA, 22), (GABP_KERNEL_TMA, 30)]
        b.iterate(-1, 0.3)
        res = b.residuals()
        assert np.all(res <= 1e-5)
        for i in (0, 17, 42, 63):
            mu, _ = b.marginals(i)
            fl = oracle_factors(orc, probs[i])
            assert orc.residual(fl, mu) <= 1.0001e-5


def test_batch_argument_errors():
    from paper_2404_12968_gb300 import (Batch, GabpError, GABP_KERNEL_FUSED, GABP_KERNEL_SWEEP,
                                        GABP_KERNEL_TMA)
    probs = gabp_synth.config_batch(seed=5, count=2, lo=32, hi=40)
    with pytest.raises(GabpError, match="FP32"):
        Batch(probs, precision=1)
    with pytest.raises(GabpError, match="strip height"):
        Batch(probs, tile_y=48)
    with pytest.raises(GabpError, match="strip height"):
        Batch(probs, kernel=GABP_KERNEL_SWEEP, tile_y=30)
    with pytest.raises(GabpError, match="30 x 22 or 30 x 30"):
        Batch(probs, kernel=GABP_KERNEL_TMA, tile_y=32)
    with pytest.raises(GabpError, match="TMA or the sweep"):
        Batch(probs, kernel=GABP_KERNEL_FUSED)
    bad = gabp_synth.config_batch(seed=5, count=2, lo=32, hi=40)
    bad[1].noise_var[0] = -1.0
    with pytest.raises(GabpError, match="problem 1"):
        Batch(bad)


def test_batched_tma_bounded_wait_reports_timeout():
    """Failure detection without a GPU fault in the batched TMA kernel: its first wait is on a
    barrier that nothing completes; the bounded wait runs out and the call reports
    GABP_ERR_TIMEOUT; a fresh batch runs normally."""
    from paper_2404_12968_gb300 import Batch, GabpError, GABP_KERNEL_TMA
    probs = gabp_synth.config_batch(seed=7, count=3, lo=40, hi=90)
    with Batch(probs, kernel=GABP_KERNEL_TMA, tile_y=30, debug_flags=1) as b:
        with pytest.raises(GabpError, match="TIMEOUT"):
            b.iterate(2, 0.3)
    with Batch(probs, kernel=GABP_KERNEL_TMA, tile_y=30) as b:
        b.iterate(2, 0.3)
        assert np.all(np.isfinite(b.residuals()))
