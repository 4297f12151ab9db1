"""Converged GaBP means against the exact posterior mean at the workloads' own sizes.

Converged loopy GaBP means equal the exact posterior mean A^-1 b (Sec. 2.3, the Weiss-Freeman
result the paper relies on).  Bars: 1e-4 relative L2 with FP32 messages (compensated belief
sums), 1e-10 with FP64 messages.  FP32: the 4096^2 benchmark workload (sampled), the 1024^2
track workload, the 2048^2 warm-start evaluation problem (sampled) and the stored instances of
the 64-instance batch (sampled, iterated as one batch); FP64: the 1024^2 track workload.

The runs stop when the means settle (relative change below 1e-7 over a chunk of iterations):
with FP32 messages the FP64 residual levels off near 5e-8 while the poorly observed smooth
modes of the small-kappa problems are still converging, so it cannot tell when to stop.

Exact means: the oracle's FP64 preconditioned conjugate gradients (``oracle.exact``), run here
for the 1024^2 workload (full-field error), and stored at 4096 seeded sample nodes by
``tests/golden/make_exact_means.py`` for the 4096^2 and 2048^2 problems and the batch instances
(sampled error over those nodes).
"""
import numpy as np
import pytest

import gabp_synth
from gpu_common import (ensure_built, golden_writer, iterate_to_floor, iterate_until_settled, load_exact_sample,
                        oracle_factors, rel_l2, same_inputs_as_sample, solver)

pytestmark = pytest.mark.gpu

GATE32, GATE64 = 1e-4, 1e-10
BETA = 0.3


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.fixture(scope="module")
def tracks_1024(orc):
    """The 1024^2 track workload and its exact mean, solved here to the PCG's rounding floor
    (the stored sample was solved the same way: checked against it)."""
    from oracle import exact
    p = gabp_synth.config_tracks_1024(0)
    fl = oracle_factors(orc, p)
    mu_ex, info = exact.exact_mean_pcg(fl, p.nx, p.ny, tol=4e-15, maxit=400)
    g = load_exact_sample("tracks_1024")
    assert same_inputs_as_sample(p, g)
    assert rel_l2(mu_ex[g["index"]], g["mean"]) < 1e-11
    return p, fl, mu_ex


def test_tracks_1024_fp64_mean_matches_exact(orc, tracks_1024):
    p, fl, mu_ex = tracks_1024
    with solver(p, "fp64") as s:
        res, its = iterate_to_floor(lambda k: s.iterate(k, BETA), s.residual, 10000, 120000)
        mu, _ = s.marginals(want_var=False)
    assert rel_l2(mu, mu_ex) < GATE64, (rel_l2(mu, mu_ex), res, its)


def test_tracks_1024_fp32_mean_matches_exact(orc, tracks_1024):
    """The 1024^2 track workload (kappa 0.05, 24 tracks) with FP32 messages: far from the tracks
    the cavity precisions fall far below the FP32 range while their information stays finite,
    the case the precision floor of the factor update exists for."""
    p, fl, mu_ex = tracks_1024
    with solver(p, "fp32") as s:
        its = iterate_until_settled(lambda k: s.iterate(k, BETA), lambda: s.marginals(want_var=False)[0],
                                    5000, 100000)
        mu, _ = s.marginals(want_var=False)
    assert rel_l2(mu, mu_ex) < GATE32, (rel_l2(mu, mu_ex), its)


def test_roofline_4096_fp32_mean_matches_exact_sampled(orc):
    """The 4096^2 benchmark workload in the benchmark's launch configuration (default kernel and
    tile), FP32 messages."""
    p = gabp_synth.config_roofline_4096(0)
    g = load_exact_sample("roofline_4096")
    assert same_inputs_as_sample(p, g)
    with solver(p, "fp32") as s:
        its = iterate_until_settled(lambda k: s.iterate(k, BETA), lambda: s.marginals(want_var=False)[0],
                                    1000, 30000)
        res = s.residual()
        mu, _ = s.marginals(want_var=False)
    fl = oracle_factors(orc, p)
    assert orc.residual(fl, mu) == pytest.approx(res, rel=1e-3)
    err = rel_l2(mu[g["index"]], g["mean"])
    assert err < GATE32, (err, res, its)


def test_warm_eval_2048_fp32_mean_matches_exact_sampled():
    """The 2048^2 warm-start evaluation problem (kappa 0.03, 48 tracks), FP32 messages."""
    p = gabp_synth.config_warm_eval(0)
    g = load_exact_sample("warm_eval_2048")
    assert same_inputs_as_sample(p, g)
    with solver(p, "fp32") as s:
        its = iterate_until_settled(lambda k: s.iterate(k, BETA), lambda: s.marginals(want_var=False)[0],
                                    5000, 100000)
        mu, _ = s.marginals(want_var=False)
    err = rel_l2(mu[g["index"]], g["mean"])
    assert err < GATE32, (err, its)


def test_batch_64_stored_instances_match_exact_sampled():
    """The 64-instance batch iterated in one launch per iteration until every instance's means
    settle: each stored instance (sides 191 to 814, kappa 0.029 to 0.096) within the FP32 bar of
    its exact mean."""
    from paper_2404_12968_gb300 import Batch
    probs = gabp_synth.config_batch(seed=0)
    stored = golden_writer().BATCH_INSTANCES
    with Batch(probs) as b:
        its = iterate_until_settled(lambda k: b.iterate(k, BETA), lambda: [b.marginals(i)[0] for i in stored],
                                    2000, 80000)
        errs = {}
        for i in stored:
            g = load_exact_sample(f"batch_{i:02d}")
            assert same_inputs_as_sample(probs[i], g), i
            errs[i] = rel_l2(b.marginals(i)[0][g["index"]], g["mean"])
    assert max(errs.values()) < GATE32, (errs, its)


def test_batch_64_per_instance_iterates_match_oracle(orc):
    """The 64-instance batch in one launch per iteration: per instance, the FP32 means after 150
    iterations against the oracle's FP64 GaBP iterates (every instance up to 300^2 nodes; the
    others' residuals against the oracle's), as for single problems."""
    from paper_2404_12968_gb300 import Batch
    probs = gabp_synth.config_batch(seed=0)
    with Batch(probs) as b:
        b.iterate(150, BETA)
        res = b.residuals()
        means = [b.marginals(i)[0] for i in range(len(probs))]
    checked = 0
    for i, p in enumerate(probs):
        fl = oracle_factors(orc, p)
        assert orc.residual(fl, means[i]) == pytest.approx(res[i], rel=1e-3), i
        if p.n <= 300 * 300:
            mu_o, _, _ = orc.gabp(fl, BETA, 150)
            assert rel_l2(means[i], mu_o) < 1e-4, (i, rel_l2(means[i], mu_o))
            checked += 1
    assert checked >= 16
