"""Pins of the oracle's early-stopping rule (oracle/early_stop.py)."""
import numpy as np
import pytest

import gabp_synth
import oracle
from oracle import early_stop as es


def test_message_change_equals_a_per_edge_loop():
    # brute force: walk every factor and slot, add |d eta| and |d Lambda|, divide by 2 E
    p = gabp_synth.make_problem(6, 5, 0.3, 2, n_uniform=7)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    _, _, m1 = oracle.gabp(fl, 0.4, 1)
    _, _, m2 = oracle.gabp(fl, 0.4, 1, messages=m1)
    total, count = 0.0, 0
    for f in range(fl.nf):
        for slot in range(int(fl.ptr[f]), int(fl.ptr[f + 1])):
            total += abs(float(m2[0][slot]) - float(m1[0][slot])) + abs(float(m2[1][slot]) - float(m1[1][slot]))
            count += 2
    assert count == 2 * fl.ne
    assert es.message_change(m2, m1) == pytest.approx(total / count, rel=1e-14)


def test_rule_stops_at_the_first_crossing():
    p = gabp_synth.config_small(0)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    t, hist, _ = es.gabp_early_stop(fl, 0.5, 1e-3, 2000)
    assert t is not None and t > 3
    ref = hist[0][1]
    assert hist[0][0] == 2
    # every earlier check was at or above the threshold; the last one below it
    assert all(d >= 1e-3 * ref for (_, d) in hist[1:-1])
    assert hist[-1] == (t, hist[-1][1]) and hist[-1][1] < 1e-3 * ref
    # the iterate is near convergence by then (the rule's purpose): here the residual is ~1e-4
    mu, _, _ = oracle.gabp(fl, 0.5, t)
    assert oracle.residual(fl, mu) < 1e-3


def test_check_every_delays_the_stop_to_the_next_check():
    p = gabp_synth.config_small(1)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    t1, _, _ = es.gabp_early_stop(fl, 0.5, 1e-3, 2000, check_every=1)
    t5, h5, _ = es.gabp_early_stop(fl, 0.5, 1e-3, 2000, check_every=5)
    assert all((tt - 2) % 5 == 0 for tt, _ in h5[1:])
    assert t1 <= t5 < t1 + 5 + 5   # monotone decay: at most the next check after t1
