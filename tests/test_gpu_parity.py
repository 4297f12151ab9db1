"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Bars (tolerances written in each test):
  * FP64 messages: the GPU iterate equals the oracle iterate to 1e-10 relative L2 (means) and
    1e-10 (variances), iteration for iteration;
  * FP32 messages (compensated beliefs): converged means within 1e-4 relative L2 of the exact
    posterior mean, variances within 1e-4 of the oracle GaBP variances;
  * the split and fused kernels give bit-identical messages;
  * full-size grids: one iteration from the GPU's own message state, recomputed by the oracle
    in FP64 over every factor, matches the GPU's next state to FP32 rounding.
"""
import numpy as np
import pytest

import gabp_synth
from gpu_common import decode_messages, ensure_built, oracle_factors, rel_l2, solver, sorted_obs_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


# ---------------------------------------------------------------------------------------
# FP64: iteration-for-iteration parity on the small configuration
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [1, 2])   # fused, split
def test_fp64_small_config_matches_oracle(orc, kernel):
    p = gabp_synth.config_small(0)
    fl = oracle_factors(orc, p)
    mu_o, var_o, _ = orc.gabp(fl, 0.5, 200)
    with solver(p, "fp64", kernel=kernel) as s:
        s.iterate(200, 0.5)
        mu, var = s.marginals()
        res = s.residual()
    assert rel_l2(mu, mu_o) < 1e-10
    assert np.max(np.abs(var - var_o) / var_o) < 1e-10
    assert res == pytest.approx(orc.residual(fl, mu), rel=1e-6)
    # error against the exact posterior after 200 iterations (reported by the bench; bounded here)
    mu_ex = orc.exact_mean(fl, p.nx)
    assert rel_l2(mu, mu_ex) < 1e-3


@pytest.mark.parametrize("shape", [(67, 45), (130, 33), (1, 1), (1, 17), (23, 1), (2, 2), (33, 8)])
def test_fp64_ragged_and_degenerate_grids(orc, shape):
    nx, ny = shape
    has_obs = nx >= 2 and ny >= 2
    p = gabp_synth.make_problem(nx, ny, 0.25, 3, n_uniform=(max(nx * ny // 6, 3) if has_obs else 0))
    if has_obs:
        # an observation exactly on the far corner, one on the origin, and a duplicate
        p.obs_x = np.concatenate([p.obs_x, [nx - 1.0, 0.0, p.obs_x[0]]])
        p.obs_y = np.concatenate([p.obs_y, [ny - 1.0, 0.0, p.obs_y[0]]])
        p.y = np.concatenate([p.y, [0.5, -0.25, p.y[0]]])
        p.noise_var = np.concatenate([p.noise_var, [0.02, 0.05, p.noise_var[0]]])
    fl = oracle_factors(orc, p)
    mu_o, var_o, _ = orc.gabp(fl, 0.5, 57)
    for kernel, tile in [(1, (32, 8)), (1, (64, 16)), (2, (0, 0))]:
        with solver(p, "fp64", kernel=kernel, tile_x=tile[0], tile_y=tile[1]) as s:
            s.iterate(57, 0.5)
            mu, var = s.marginals()
        if has_obs:
            assert rel_l2(mu, mu_o) < 1e-10, (kernel, tile)
        else:
            assert np.all(mu == 0.0)
        assert np.max(np.abs(var - var_o) / var_o) < 1e-10, (kernel, tile)
    if nx == 1 and ny == 1:
        # a single cell factor with coefficient kappa^2: Lambda = kappa^4
        assert var[0] == pytest.approx(1.0 / 0.25 ** 4, rel=1e-12)


def test_fp64_paper_init_and_gamma(orc):
    p = gabp_synth.make_problem(40, 31, 0.3, 5, n_uniform=150)
    fl = orc.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, 2.5)
    mu_o, var_o, _ = orc.gabp(fl, 0.4, 90, init="paper")
    with solver(p, "fp64", gamma=2.5, init=1) as s:
        s.iterate(90, 0.4)
        mu, var = s.marginals()
    assert rel_l2(mu, mu_o) < 1e-10
    assert np.max(np.abs(var - var_o) / var_o) < 1e-10


def test_fp64_warm_start_matches_oracle(orc):
    p = gabp_synth.make_problem(48, 40, 0.2, 8, n_uniform=200)
    fl = oracle_factors(orc, p)
    rng = np.random.default_rng(1)
    mu0 = p.truth.reshape(-1) + 0.1 * rng.standard_normal(p.n)
    lam0 = rng.uniform(0.5, 5.0, p.n)
    with solver(p, "fp64") as s:
        s.warm_start(mu0, lam0)
        mu, var = s.marginals()
        np.testing.assert_allclose(mu, mu0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(var, 1.0 / lam0, rtol=1e-12)
        s.iterate(75, 0.5)
        mu, var = s.marginals()
    mu_o, var_o, _ = orc.gabp(fl, 0.5, 75, init="warm", mu0=mu0, lam0=lam0)
    assert rel_l2(mu, mu_o) < 1e-10
    assert np.max(np.abs(var - var_o) / var_o) < 1e-10


# ---------------------------------------------------------------------------------------
# split and fused kernels: identical arithmetic, identical bits
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(67, 45), (68, 45), (256, 130), (300, 7), (4, 2), (4, 37), (124, 1), (32, 15)])
def test_split_and_fused_bit_identical(prec, shape):
    """Every kernel and tile shape gives the same bits; includes the narrowest TMA grid (4
    columns), a single row without observations and tiles ragged in both directions."""
    nx, ny = shape
    obs = nx >= 2 and ny >= 2
    p = gabp_synth.make_problem(nx, ny, 0.05, 9, n_tracks=4 if obs else 0, per_track=nx,
                                n_uniform=max(nx * ny // 20, 2) if obs else 0, sigma=(0.02, 0.1))
    variants = [(2, (0, 0)), (1, (32, 8)), (1, (64, 16)), (1, (128, 8)), (1, (32, 32))]
    if prec == "fp32" and nx % 4 == 0:
        # TMA tiles, each with runs of 1 (no belief rows reused) and longer runs (ragged last band)
        variants += [(3, (30, 14), 1), (3, (30, 14), 2), (3, (30, 14), 3), (3, (30, 14), 8), (3, (30, 22), 1),
                     (3, (30, 22), 4), (3, (30, 30), 1), (3, (30, 30), 5)]
    if prec == "fp32":
        variants += [(4, (30, 16)), (4, (30, 32)), (4, (30, 64)), (4, (30, 128))]
    bufs = []
    for kernel, tile, *run in variants:
        with solver(p, prec, kernel=kernel, tile_x=tile[0], tile_y=tile[1], tile_run=run[0] if run else 0) as s:
            s.iterate(41, 0.3)        # odd: exercises the ping-pong parity and the graph chunking
            bufs.append(s.get_messages())
    for b in bufs[1:]:
        assert np.array_equal(b, bufs[0])


def test_tma_tile_runs():
    """The TMA schedule's run length: chosen in 1..4 by default, settable in 1..8, reported by the
    stats, refused outside 0..8; every length gives the bits of runs of 1 at a size with
    thousands of tiles."""
    p = gabp_synth.make_problem(1024, 700, 0.05, 3, n_tracks=8, per_track=1024, n_uniform=20000)
    bufs = []
    for run in (0, 1, 4, 7):
        with solver(p, "fp32", kernel=3, tile_run=run) as s:
            st = s.stats()
            assert 1 <= st["tile_run"] <= (4 if run == 0 else run) and (run == 0 or st["tile_run"] == run)
            s.iterate(25, 0.3)
            bufs.append(s.get_messages())
    for b in bufs[1:]:
        assert np.array_equal(b, bufs[0])
    from paper_2404_12968_gb300 import GabpError
    with solver(p, "fp32", kernel=2) as s:
        assert s.stats()["tile_run"] == 0
    with pytest.raises(GabpError):
        solver(p, "fp32", kernel=3, tile_run=9)


def test_deterministic_repeat():
    p = gabp_synth.config_small(2)
    outs = []
    for _ in range(2):
        with solver(p, "fp32") as s:
            s.iterate(123, 0.5)
            outs.append((s.get_messages(), s.residual()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_checkpoint_resume():
    p = gabp_synth.config_small(1)
    with solver(p, "fp32") as s:
        s.iterate(30, 0.5)
        ck = s.get_messages()
        s.iterate(25, 0.5)
        a = s.get_messages()
        s.set_messages(ck)
        s.iterate(25, 0.5)
        b = s.get_messages()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------------------
# FP32 messages with compensated beliefs
# ---------------------------------------------------------------------------------------

def test_fp32_small_config_tracks_oracle(orc):
    p = gabp_synth.config_small(0)
    fl = oracle_factors(orc, p)
    for its in (10, 200):
        mu_o, var_o, _ = orc.gabp(fl, 0.5, its)
        with solver(p, "fp32") as s:
            s.iterate(its, 0.5)
            mu, var = s.marginals()
        assert rel_l2(mu, mu_o) < 1e-5
        assert np.max(np.abs(var - var_o) / var_o) < 1e-5


@pytest.mark.parametrize("kappa,seed", [(0.05, 0), (0.02, 1)])
def test_fp32_converged_mean_matches_exact(orc, kappa, seed):
    """Converged FP32 GaBP mean vs the exact posterior mean, in the configurations' small-kappa,
    track-observed regime at a size the band solver handles.  Iterate until the FP64 residual
    stops improving (the FP32 floor), then gate the mean at 1e-4 relative L2."""
    p = gabp_synth.scaled_config(192, kappa, 700 + seed, 10, n_uniform=300, sigma=(0.02, 0.1))
    fl = oracle_factors(orc, p)
    mu_ex = orc.exact_mean(fl, p.nx)
    with solver(p, "fp32") as s:
        best = np.inf
        for _ in range(40):
            s.iterate(2000, 0.3)
            res = s.residual()
            if res > 0.5 * best:
                break
            best = min(best, res)
        mu, var = s.marginals()
        res = s.residual()
    assert orc.residual(fl, mu) == pytest.approx(res, rel=1e-3)
    assert res < 1e-6
    assert rel_l2(mu, mu_ex) < 1e-4, (rel_l2(mu, mu_ex), res)
    # variances: the precision recursion does not involve the means and settles early;
    # compare with the oracle GaBP variances once those have settled
    _, var_a, _ = orc.gabp(fl, 0.3, 1500)
    _, var_b, _ = orc.gabp(fl, 0.3, 2000)
    assert np.max(np.abs(var_a - var_b) / var_b) < 1e-9
    assert np.max(np.abs(var - var_b) / var_b) < 1e-4


def test_tracks_1024_reaches_residual_and_oracle_agrees(orc):
    p = gabp_synth.config_tracks_1024(0)
    fl = oracle_factors(orc, p)
    with solver(p, "fp32", tol=1e-5) as s:
        s.iterate(-1, 0.3)
        mu, _ = s.marginals(want_var=False)
        res = s.residual()
    assert res <= 1e-5
    assert orc.residual(fl, mu) <= 1.0001e-5


# ---------------------------------------------------------------------------------------
# full-size one-step parity
# ---------------------------------------------------------------------------------------

def _gpu_state_to_oracle_slots(orc, p, fl, prior, obs):
    """Map the GPU message buffer onto the oracle's factor-list slots (cell factors first, slot
    order self, W, E, S, N; then observations in input order, corners in weight order)."""
    nx, ny, n = p.nx, p.ny, p.n
    ii, jj = np.divmod(np.arange(n), nx)
    exists = np.stack([np.ones(n, bool), jj > 0, jj < nx - 1, ii > 0, ii < ny - 1], axis=1)
    pe = prior[:, :, 0].T[exists].astype(np.float64)
    pl = prior[:, :, 1].T[exists].astype(np.float64)
    order, _, _ = sorted_obs_order(orc, p)
    oe = np.empty((p.m, 4))
    ol = np.empty((p.m, 4))
    oe[order] = obs[:, :, 0]
    ol[order] = obs[:, :, 1]
    me = np.concatenate([pe, oe.reshape(-1)])
    ml = np.concatenate([pl, ol.reshape(-1)])
    assert me.shape[0] == fl.ne
    return me, ml


@pytest.mark.parametrize("cfg", ["tracks_1024", "roofline_4096"])
def test_full_size_one_step_parity(orc, cfg):
    p = getattr(gabp_synth, f"config_{cfg}")(0)
    fl = oracle_factors(orc, p)
    beta = 0.3
    with solver(p, "fp32") as s:     # the fused kernel with the default tile: the benchmarked launch
        s.iterate(20, beta)
        t0 = s.get_messages()
        s.iterate(1, beta)
        t1 = s.get_messages()
    me0, ml0 = _gpu_state_to_oracle_slots(orc, p, fl, *decode_messages(t0, p))
    me1, ml1 = _gpu_state_to_oracle_slots(orc, p, fl, *decode_messages(t1, p))
    _, _, (me_o, ml_o) = orc.gabp(fl, beta, 1, messages=(me0, ml0))
    assert rel_l2(ml1, ml_o) < 2e-6
    assert rel_l2(me1, me_o) < 2e-5
    # element-wise, relative to each message type's scale
    scale_l = np.abs(ml_o).mean()
    scale_e = np.abs(me_o).mean()
    assert np.max(np.abs(ml1 - ml_o) / (np.abs(ml_o) + scale_l)) < 1e-4
    assert np.max(np.abs(me1 - me_o) / (np.abs(me_o) + scale_e)) < 1e-3


# ---------------------------------------------------------------------------------------
# argument errors become status codes
# ---------------------------------------------------------------------------------------

def test_argument_errors():
    from paper_2404_12968_gb300 import GabpError, Solver
    p = gabp_synth.make_problem(16, 12, 0.3, 0, n_uniform=10)
    xy = np.stack([p.obs_x, p.obs_y], 1)
    bad = [
        dict(kappa=0.0), dict(kappa=-1.0), dict(kappa=float("nan")),
    ]
    for b in bad:
        with pytest.raises(GabpError, match="ARG"):
            Solver(nx=16, ny=12, kappa=b["kappa"], obs_xy=xy, y=p.y, noise_var=p.noise_var)
    xy2 = xy.copy()
    xy2[3, 0] = 15.0 + 1e-9
    with pytest.raises(GabpError, match="outside"):
        Solver(nx=16, ny=12, kappa=0.3, obs_xy=xy2, y=p.y, noise_var=p.noise_var)
    nv = p.noise_var.copy()
    nv[0] = 0.0
    with pytest.raises(GabpError, match="ARG"):
        Solver(nx=16, ny=12, kappa=0.3, obs_xy=xy, y=p.y, noise_var=nv)
    yy = p.y.copy()
    yy[1] = np.inf
    with pytest.raises(GabpError, match="ARG"):
        Solver(nx=16, ny=12, kappa=0.3, obs_xy=xy, y=yy, noise_var=p.noise_var)
    with pytest.raises(GabpError, match="ARG"):
        Solver(nx=16, ny=12, kappa=0.3, obs_xy=xy, y=p.y, noise_var=p.noise_var, tile_x=48, tile_y=8)
    with pytest.raises(GabpError, match="ARG"):
        Solver(nx=1, ny=12, kappa=0.3, obs_xy=np.zeros((1, 2)), y=np.zeros(1), noise_var=np.ones(1))
    with Solver(p) as s:
        with pytest.raises(GabpError, match="damping"):
            s.iterate(3, 1.0)
        with pytest.raises(GabpError, match="damping"):
            s.iterate(3, -0.1)
        s.iterate(3, 0.5)   # the context stays usable after an argument error


def test_auto_kernel_selection():
    from paper_2404_12968_gb300 import GABP_KERNEL_FUSED, GABP_KERNEL_SWEEP, GABP_KERNEL_TMA
    for (nx, prec, expect) in [(64, "fp32", GABP_KERNEL_TMA), (66, "fp32", GABP_KERNEL_SWEEP),
                               (64, "fp64", GABP_KERNEL_FUSED)]:
        p = gabp_synth.make_problem(nx, 40, 0.3, 0, n_uniform=50)
        with solver(p, prec) as s:
            assert s.stats()["kernel"] == expect


def test_kernel_bounded_wait_reports_timeout():
    """Failure detection without a GPU fault: the TMA kernel's first wait is on a barrier that
    nothing completes; the bounded wait runs out, the status is GABP_ERR_TIMEOUT, the messages are
    untouched and the context stays usable."""
    from paper_2404_12968_gb300 import GabpError, GABP_KERNEL_TMA
    p = gabp_synth.config_small(0)
    with solver(p, "fp32", kernel=GABP_KERNEL_TMA, debug_flags=1) as s:
        before = s.get_messages()
        with pytest.raises(GabpError, match="TIMEOUT"):
            s.iterate(3, 0.5)
        assert np.array_equal(s.get_messages(), before)
        assert s.stats()["iterations"] == 0
        assert np.isfinite(s.residual())
    with solver(p, "fp32", kernel=GABP_KERNEL_TMA) as s:   # a fresh context runs normally
        s.iterate(3, 0.5)


def test_iterate_timeout_status():
    from paper_2404_12968_gb300 import GabpError
    p = gabp_synth.config_tracks_1024(0)
    with solver(p, "fp32", tol=1e-12, check_every=10, max_iters=30) as s:
        with pytest.raises(GabpError, match="TIMEOUT"):
            s.iterate(-1, 0.3)
        assert s.stats()["iterations"] == 30
        s.iterate(2, 0.3)
