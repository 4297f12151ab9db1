"""Grid spacing h of the prior's Laplacian (App. C's finite differences at spacing h; the
paper's synthetic setting discretises the unit square with h = 1 / N).  The library works at
unit spacing internally (L_h = h^-2 L_1(kappa h)); the oracle builds L_h directly."""
import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("alpha,h", [(2, 0.25), (2, 3.0), (4, 0.5)])
def test_fp64_iterates_with_grid_spacing_match_oracle(orc, alpha, h):
    from paper_2404_12968_gb300 import Solver
    p = gabp_synth.scaled_config(40, 0.4, 1, 3, n_uniform=60)
    gamma = 0.7
    beta = 0.5
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, gamma, alpha, h=h)
    mu_o, var_o, _ = orc.gabp(fl, beta, 60)
    with Solver(p, precision="fp64", gamma=gamma, alpha=alpha, h=h) as s:
        s.iterate(60, beta)
        mu, var = s.marginals()
        res = s.residual()
    assert rel_l2(mu, mu_o) < 1e-10
    assert rel_l2(var, var_o) < 1e-10
    assert res == pytest.approx(orc.residual(fl, mu), rel=1e-9)


def test_spacing_is_the_rescaled_unit_spacing_prior():
    """h = 0.5 (exact powers of two) against h = 1 with kappa h and gamma / h^4: the same
    factors, so the same messages bit for bit."""
    from paper_2404_12968_gb300 import Solver
    p = gabp_synth.scaled_config(48, 0.1, 2, 4, n_uniform=100)
    h = 0.5
    with Solver(p, precision="fp32", gamma=1.3, h=h) as a, \
            Solver(nx=p.nx, ny=p.ny, kappa=p.kappa * h, obs_xy=np.stack([p.obs_x, p.obs_y], 1), y=p.y,
                   noise_var=p.noise_var, precision="fp32", gamma=1.3 / h ** 4) as b:
        a.iterate(40, 0.3)
        b.iterate(40, 0.3)
        assert np.array_equal(a.get_messages(), b.get_messages())


def test_spacing_refused_when_not_positive():
    from paper_2404_12968_gb300 import GabpError, Solver
    p = gabp_synth.scaled_config(16, 0.3, 0, 1)
    for h in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(GabpError, match="spacing"):
            Solver(p, precision="fp32", h=h)
