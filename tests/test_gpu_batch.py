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


def test_batch_lockstep_bit_identical_to_single_contexts():
    from paper_2404_12968_gb300 import Batch, GABP_KERNEL_SWEEP
    probs = gabp_synth.config_batch(seed=3, count=6, lo=48, hi=200)
    with Batch(probs, tile_y=32) as b:
        assert b.strip_height == 32
        b.iterate(37, 0.3)
        means = [b.marginals(i)[0] for i in range(len(probs))]
        for i, p in enumerate(probs):
            with solver(p, "fp32", kernel=GABP_KERNEL_SWEEP, tile_x=30, tile_y=32) as s:
                s.iterate(37, 0.3)
                mu, _ = s.marginals(want_var=False)
            assert np.array_equal(mu, means[i]), i
            assert b.stats(i)["iterations"] == 37


def test_batch_until_tolerance_matches_oracle_residual(orc):
    from paper_2404_12968_gb300 import Batch
    probs = gabp_synth.config_batch(seed=4, count=10, lo=64, hi=256)
    with Batch(probs, tol=1e-5, check_every=20) as b:
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
    from paper_2404_12968_gb300 import Batch
    probs = gabp_synth.config_batch(seed=0)
    assert len(probs) == 64
    with Batch(probs, tol=1e-5) as b:
        assert b.strip_height in (16, 32, 64, 128)
        b.iterate(-1, 0.3)
        res = b.residuals()
        assert np.all(res <= 1e-5)
        for i in (0, 17, 42, 63):
            mu, _ = b.marginals(i)
            fl = oracle_factors(orc, probs[i])
            assert orc.residual(fl, mu) <= 1.0001e-5


def test_batch_argument_errors():
    from paper_2404_12968_gb300 import Batch, GabpError
    probs = gabp_synth.config_batch(seed=5, count=2, lo=32, hi=40)
    with pytest.raises(GabpError, match="FP32"):
        Batch(probs, precision=1)
    with pytest.raises(GabpError, match="strip height"):
        Batch(probs, tile_y=48)
    bad = gabp_synth.config_batch(seed=5, count=2, lo=32, hi=40)
    bad[1].noise_var[0] = -1.0
    with pytest.raises(GabpError, match="problem 1"):
        Batch(bad)
