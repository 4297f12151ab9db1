"""The paper's early-stopping rule on the GPU against the oracle's (oracle/early_stop.py)."""
import pytest

import gabp_synth
from gpu_common import ensure_built, oracle_factors, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_fp64_message_change_matches_oracle(orc):
    from oracle import early_stop as es
    p = gabp_synth.config_small(2)
    fl = oracle_factors(orc, p)
    msg = orc.init_messages(fl, "cold")
    with solver(p, "fp64") as s:
        done = 0
        for k in (1, 1, 5, 30):
            prev = msg
            if k > 1:
                _, _, prev = orc.gabp(fl, 0.5, k - 1, messages=msg)
            _, _, msg = orc.gabp(fl, 0.5, 1, messages=prev)
            s.iterate(k, 0.5)
            done += k
            assert s.message_change() == pytest.approx(es.message_change(msg, prev), rel=1e-10), done


@pytest.mark.parametrize("seed", [0, 1])
def test_fp64_stops_at_the_oracles_iteration(orc, seed):
    from oracle import early_stop as es
    p = gabp_synth.config_small(seed)
    fl = oracle_factors(orc, p)
    t_o, hist, _ = es.gabp_early_stop(fl, 0.5, 1e-3, 2000)
    # the decision is not on a knife edge at the stopping check
    assert hist[-1][1] < 0.999e-3 * hist[0][1] and hist[-2][1] > 1.001e-3 * hist[0][1]
    with solver(p, "fp64") as s:
        t = s.iterate_early_stop(2000, 0.5, 1e-3, 1)
        assert s.stats()["iterations"] == t
    assert t == t_o


def test_fp32_rule_with_a_coarser_check(orc):
    p = gabp_synth.scaled_config(128, 0.1, 4, 6)
    with solver(p, "fp32") as s:
        t = s.iterate_early_stop(20000, 0.3, 1e-3, 10)
        assert (t - 2) % 10 == 0 and t > 12
        d_stop = s.message_change()
        s.reset()
        s.iterate(2, 0.3)
        ref = s.message_change()
        assert d_stop < 1e-3 * ref
        s.reset()
        s.iterate(t - 10, 0.3)
        assert s.message_change() >= 1e-3 * ref   # the previous check had not stopped


def test_early_stop_argument_and_state_errors():
    from paper_2404_12968_gb300 import GabpError
    p = gabp_synth.config_small(0)
    with solver(p, "fp32") as s:
        with pytest.raises(GabpError):
            s.message_change()                   # no iteration yet
        for args in [(2, 0.5, 1e-3, 1), (100, 0.5, 0.0, 1), (100, 0.5, 1e-3, 0), (100, 1.0, 1e-3, 1)]:
            with pytest.raises(GabpError):
                s.iterate_early_stop(*args)
        with pytest.raises(GabpError) as e:
            s.iterate_early_stop(4, 0.5, 1e-12, 1)   # max_iters first
        assert e.value.code == 5
