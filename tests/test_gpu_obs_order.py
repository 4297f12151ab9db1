"""The observation layout that gabp_create builds on the GPU: base cells and the stable sort of
the observations by base cell (ties in input order), the order of the observation messages in
the message buffer.  Pinned against the oracle's bilinear rule and numpy's stable argsort on
problems with heavy ties: thousands of observations in one cell (more than one sort chunk),
ties spread over chunk boundaries, observations on the last grid lines (clamped base cells),
and grids whose cell count needs one, two and three radix passes."""
import numpy as np
import pytest

import gabp_synth
from gpu_common import decode_messages, ensure_built, rel_l2, solver, sorted_obs_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _tied_problem(nx, ny, m, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, nx - 1, m)
    y = rng.uniform(0, ny - 1, m)
    # a third of the observations in one cell, a tenth in a handful of cells, some on the last
    # grid lines (their base cell is clamped to the last full cell)
    a = m // 3
    x[:a] = min(1, nx - 2) + 0.999 * rng.uniform(0, 1, a)
    y[:a] = min(2, ny - 2) + 0.999 * rng.uniform(0, 1, a)
    b = a + m // 10
    cells = rng.integers(0, 6, b - a)
    x[a:b] = np.minimum((cells % 3) + 0.25 + 0.5 * rng.uniform(0, 1, b - a), nx - 1)
    y[a:b] = (ny - 2) + 0.5 * (cells // 3) * rng.uniform(0, 1, b - a)
    x[b:b + 50] = nx - 1.0
    y[b + 50:b + 100] = ny - 1.0
    perm = rng.permutation(m)   # spread the tied groups over the input order
    x, y = x[perm], y[perm]
    noise = rng.uniform(0.01, 0.2, m)   # distinct: each observation recognisable by its Lambda
    return gabp_synth.Problem(nx, ny, 0.3, x, y, rng.normal(size=m), noise)


@pytest.mark.parametrize("nx,ny,m", [(9, 7, 5000), (70, 50, 9000), (300, 250, 20000), (2, 2, 3000)])
def test_observation_messages_in_stable_base_order(orc, nx, ny, m):
    """Cold-start observation messages are (0, w_c^2 / sigma^2) per corner: decoded from the
    buffer, they must follow the oracle's stable order of the observations by base cell."""
    p = _tied_problem(nx, ny, m, seed=nx * 7 + m)
    order, base, w = sorted_obs_order(orc, p)
    with solver(p, "fp64") as s:
        _, obs = decode_messages(s.get_messages(), p, "fp64")
    expect = (w ** 2 / p.noise_var[:, None])[order]
    assert np.all(obs[:, :, 0] == 0.0)
    np.testing.assert_allclose(obs[:, :, 1], expect, rtol=1e-12, atol=0)


def test_tied_problem_iterates_match_oracle(orc):
    """Iterates on a tie-heavy problem against the oracle's GaBP (the observation index and the
    message order agree with each other)."""
    from gpu_common import oracle_factors
    p = _tied_problem(40, 30, 4000, seed=5)
    fl = oracle_factors(orc, p)
    mu0, var0, _ = orc.gabp(fl, 0.5, 30)
    with solver(p, "fp64") as s:
        s.iterate(30, 0.5)
        mu, var = s.marginals()
    assert rel_l2(mu, mu0) < 1e-10
    assert np.max(np.abs(var - var0) / var0) < 1e-10


def test_invalid_observations_rejected_while_the_gpu_sorts():
    """Creation validates the observations on the host while the GPU copies and sorts them: the
    first invalid index decides the error, nothing faults on the invalid values (NaN, negative
    or out-of-grid coordinates, zero variance), and a valid problem afterwards is unaffected."""
    from paper_2404_12968_gb300 import GabpError
    p = _tied_problem(70, 50, 9000, seed=3)
    cases = []
    x = p.obs_x.copy(); x[4321] = np.nan
    cases.append((x, p.obs_y, p.noise_var, "non-finite observation data at index 4321"))
    x = p.obs_x.copy(); x[17] = -3.0; x[5000] = 1e9
    cases.append((x, p.obs_y, p.noise_var, "observation 17 outside the grid"))
    v = p.noise_var.copy(); v[8999] = 0.0
    cases.append((p.obs_x, p.obs_y, v, "noise variance must be > 0"))
    for ox, oy, nv, msg in cases:
        q = gabp_synth.Problem(p.nx, p.ny, p.kappa, ox, oy, p.y, nv)
        with pytest.raises(GabpError, match=msg):
            solver(q, "fp64")
    with solver(p, "fp64") as s:
        s.iterate(5, 0.5)
        assert np.isfinite(s.residual())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_marginals_into_pinned_host_memory(precision):
    """gabp_marginals writes into pinned host buffers through their device address, into other
    host buffers through a staging copy, and into device buffers directly: the same values."""
    import torch
    from paper_2404_12968_gb300 import gabp_marginals
    p = _tied_problem(70, 50, 3000, seed=8)
    with solver(p, precision) as s:
        s.iterate(20, 0.5)
        ref_m, ref_v = s.marginals()                        # pageable numpy arrays
        pm = torch.empty(p.n, dtype=torch.float64, pin_memory=True)
        pv = torch.empty(p.n, dtype=torch.float64, pin_memory=True)
        gabp_marginals(s.ctx, pm.numpy(), pv.numpy())
        assert np.array_equal(pm.numpy(), ref_m) and np.array_equal(pv.numpy(), ref_v)
        pm2 = torch.empty(p.n, dtype=torch.float64, pin_memory=True)
        v2 = np.empty(p.n)                                  # pinned mean, pageable variance
        gabp_marginals(s.ctx, pm2.numpy(), v2)
        assert np.array_equal(pm2.numpy(), ref_m) and np.array_equal(v2, ref_v)
        dm = torch.empty(p.n, dtype=torch.float64, device="cuda")
        gabp_marginals(s.ctx, dm, None)
        assert np.array_equal(dm.cpu().numpy(), ref_m)
