"""The multigrid warm start on the GPU against the oracle's (oracle/multigrid.py)."""
import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built, oracle_factors, rel_l2, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _oracle_mg(p, levels, beta, iters):
    from oracle import multigrid as mg
    return mg.multigrid_init(p.nx, p.ny, p.kappa, 1.0, p.obs_x, p.obs_y, p.y, p.noise_var, levels, beta, iters)


@pytest.mark.parametrize("shape,levels", [((67, 45), 3), ((64, 48), 4)])
def test_fp64_fixed_iterations_match_oracle(shape, levels):
    """Every level runs a fixed number of iterations: the target's initial marginals, and every
    level's residual and damping, equal the oracle's."""
    from paper_2404_12968_gb300 import Multigrid
    nx, ny = shape
    p = gabp_synth.make_problem(nx, ny, 0.1, 5, n_uniform=nx * ny // 12, n_tracks=2, per_track=nx, sigma=(0.05, 0.1))
    mu0, lam0, info = _oracle_mg(p, levels, 0.3, 80)
    with solver(p, "fp64") as s:
        with Multigrid(s, levels) as mg:
            st = mg.warm_start(0.3, 0.0, 80)
        mu, var = s.marginals()
        assert s.stats()["iterations"] == 0
    assert rel_l2(mu, mu0) < 1e-10
    assert np.max(np.abs(1.0 / var - lam0) / lam0) < 1e-10
    for k in range(1, levels):
        r, b, ok = info[k]
        assert st["converged"][k] == ok and st["damping"][k] == pytest.approx(b)
        assert st["residual"][k] == pytest.approx(r, rel=1e-6)
        assert st["iterations"][k] == 80


def test_fp64_diverging_coarse_level_is_rerun_with_more_damping():
    """40 observations on an 8 x 8 coarsest level: GaBP diverges there at damping 0.3 and the
    level is re-run at 0.65, as in the oracle."""
    from paper_2404_12968_gb300 import Multigrid
    p = gabp_synth.make_problem(64, 64, 0.05, 4, n_uniform=40, n_tracks=0, per_track=0, sigma=(0.05, 0.05))
    mu0, lam0, info = _oracle_mg(p, 4, 0.3, 300)
    with solver(p, "fp64") as s:
        with Multigrid(s, 4) as mg:
            st = mg.warm_start(0.3, 0.0, 300)
        mu, var = s.marginals()
    assert st["damping"][3] == pytest.approx(0.65) and st["converged"][3]
    assert st["iterations"][3] == 600   # the diverged run and the re-run
    assert st["damping"][2] == pytest.approx(0.3) and st["damping"][1] == pytest.approx(0.3)
    assert rel_l2(mu, mu0) < 1e-9
    assert np.max(np.abs(1.0 / var - lam0) / lam0) < 1e-9


def test_fp32_multigrid_reaches_tolerance_in_fewer_fine_iterations(orc):
    """FP32, levels iterated to the tolerance: the target then needs fewer iterations to relative
    residual 1e-5 than from the cold start, and the oracle confirms the final residual."""
    from paper_2404_12968_gb300 import Multigrid
    p = gabp_synth.scaled_config(256, 0.03, 11, 8)
    with solver(p, "fp32", tol=1e-5, check_every=10, max_iters=100000) as s:
        s.iterate(-1, 0.3)
        cold = s.stats()["iterations"]
        with Multigrid(s, 4) as mg:
            st = mg.warm_start(0.3, 1e-5, 20000)
            assert all(st["converged"][1:])
            assert all(r <= 1e-5 for r in st["residual"][1:])
            s.iterate(-1, 0.3)
            warm = s.stats()["iterations"]
            res = s.residual()
            mu, _ = s.marginals(want_var=False)
    assert res <= 1e-5
    assert warm < cold, (warm, cold)
    fl = oracle_factors(orc, p)
    assert orc.residual(fl, mu) == pytest.approx(res, rel=1e-3)


def test_multigrid_argument_errors():
    from paper_2404_12968_gb300 import GabpError, Multigrid
    p = gabp_synth.make_problem(20, 12, 0.2, 1, n_uniform=30)
    with solver(p, "fp32") as s:
        with pytest.raises(GabpError):
            Multigrid(s, 1)
        with pytest.raises(GabpError):
            Multigrid(s, 5)            # level 4 would have 2 x 1 nodes
        with pytest.raises(GabpError):
            Multigrid(s, 17)
        with Multigrid(s, 2) as mg:
            with pytest.raises(GabpError):
                mg.warm_start(1.0, 1e-5, 100)
            with pytest.raises(GabpError):
                mg.warm_start(0.3, 1e-5, 0)
