"""What the trained warm-start network gains over plain GaBP without it.

The shipped weights (``paper_2404_12968_gb300/weights/wsnet_512.npy``) were trained on the GPU
by the library's own kernels on 2000 plain-GaBP posteriors at 512^2.  On the 2048^2 evaluation
problem (kappa 0.03, 48 tracks, never seen in training) the learned warm start must reach the
relative residual 1e-5 in fewer iterations and less wall time than the cold start, network
inference included; an untrained network of the same shape must not do as well as the trained
one; the oracle confirms every final residual.  The plain cold start is the method without the
network; the multigrid warm start (Sec. 3.2) is reported beside them by the benchmark.
"""
import os

import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built, oracle_factors

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2404_12968_gb300",
                       "weights", "wsnet_512.npy")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_trained_warm_start_beats_cold_start_and_untrained_network(orc):
    from paper_2404_12968_gb300 import Solver, WarmStartNet
    from paper_2404_12968_gb300.warmstart import DAMPING, TOL, time_to_tol
    p = gabp_synth.config_warm_eval(0)
    fl = oracle_factors(orc, p)
    trained = WarmStartNet(seed=0, device=0)
    trained.load(WEIGHTS)
    untrained = WarmStartNet(seed=0, device=0)
    try:
        with Solver(p, precision="fp32", tol=TOL, check_every=10, max_iters=400000) as s:
            time_to_tol(s, None)          # warm-up: graph capture, first launches
            time_to_tol(s, trained)
            cold = min((time_to_tol(s, None) for _ in range(3)), key=lambda r: r[0])
            mu_cold, _ = s.marginals(want_var=False)
            warm = min((time_to_tol(s, trained) for _ in range(3)), key=lambda r: r[0])
            mu_warm, _ = s.marginals(want_var=False)
            plain = time_to_tol(s, untrained)
    finally:
        trained.close()
        untrained.close()
    (c_s, c_it, c_res, _), (w_s, w_it, w_res, _), (_, u_it, _, _) = cold, warm, plain
    assert c_res <= TOL and w_res <= TOL
    # the oracle's FP64 residual of both final means
    assert orc.residual(fl, mu_cold) <= 1.001 * TOL
    assert orc.residual(fl, mu_warm) <= 1.001 * TOL
    # the gain: fewer iterations and less wall time with the trained network (inference included)
    assert w_it < 0.6 * c_it, (w_it, c_it)
    assert w_s < c_s, (w_s, c_s)
    # training is what makes the difference
    assert w_it < u_it, (w_it, u_it)
    assert DAMPING == 0.3
