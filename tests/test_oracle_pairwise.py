"""Pins of the oracle's pairwise re-weighted message passing (oracle/pairwise.py)."""
import numpy as np
import pytest

import gabp_synth
import oracle
from oracle import pairwise as pw


def _grid_point_problem(N, kappa, frac, seed=0, sigma=0.1):
    """Observations at a fraction of the grid points (the paper's synthetic setting)."""
    rng = np.random.default_rng(seed)
    nobs = int(frac * N * N)
    idx = rng.choice(N * N, nobs, replace=False)
    p = gabp_synth.make_problem(N, N, kappa, seed + 1)
    y = p.truth.reshape(-1)[idx] + sigma * rng.standard_normal(nobs)
    ox = (idx % N).astype(float)
    oy = (idx // N).astype(float)
    return oracle.build_factors(N, N, kappa, ox, oy, y, np.full(nobs, sigma ** 2))


@pytest.mark.parametrize("c", [1.0, 10.0, -2.0, 0.5])
def test_factor_message_equals_the_fractional_integral(c):
    # m^(1/c)(f) = integral of exp(-(P/c) f g) exp(-alpha g^2 / 2 + beta g) dg, by quadrature:
    # its log is a quadratic in f whose coefficients must be (-a/2, b)
    alpha, beta, pij = 2.7, -0.8, -1.3
    a, b = pw.factor_message(alpha, beta, pij, c)
    g = np.linspace(-40, 40, 400001)
    fs = np.array([-0.7, -0.2, 0.3, 0.9])
    logI = []
    for f in fs:
        e = -(pij / c) * f * g - 0.5 * alpha * g * g + beta * g
        m = e.max()
        logI.append(m + np.log(np.trapezoid(np.exp(e - m), g)))
    coef = np.polyfit(fs, np.array(logI), 2)
    assert coef[0] == pytest.approx(-0.5 * a, rel=1e-6, abs=1e-9)
    assert coef[1] == pytest.approx(b, rel=1e-6, abs=1e-9)


def test_assembled_precision_is_the_posterior_precision():
    p = gabp_synth.make_problem(9, 7, 0.4, 3, n_uniform=15)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    P, h = pw.assemble(fl)
    np.testing.assert_allclose(P.toarray(), oracle.dense_A(fl), rtol=1e-13, atol=1e-13)
    # interior rows of gamma L^T L have the 13-point pattern; bilinear observations stay inside it
    src, dst, _, rev = pw.edges(P)
    assert np.bincount(dst, minlength=fl.n).max() == 12
    assert np.array_equal(src[rev], dst) and np.array_equal(dst[rev], src)


@pytest.mark.parametrize("c", [10.0, 20.0])
def test_converged_means_are_exact(c):
    # a fixed point of the re-weighted scheme carries the exact posterior means
    fl = _grid_point_problem(32, 0.3, 0.05)
    P, h = pw.assemble(fl)
    exact = oracle.exact_mean(fl, 32)
    mean, prec, _, ok = pw.run(P, h, c, 0.6, 20000)
    assert ok and np.all(prec > 0)
    assert np.linalg.norm(mean - exact) / np.linalg.norm(exact) < 1e-9


def test_reproduces_the_papers_convergence_pattern():
    # the grid search of App. D (5 % of the grid observed, learning rate 0.6): c = 1 and c = 5
    # diverge, c = 10 and c = 20 converge; learning rate 0.8 diverges for c = 10
    fl = _grid_point_problem(64, 0.05, 0.05)
    P, h = pw.assemble(fl)
    exact = oracle.exact_mean(fl, 64)

    def diverged(c, eta):
        mean, _, _, ok = pw.run(P, h, c, eta, 2000)
        return not ok or not np.linalg.norm(mean - exact) / np.linalg.norm(exact) < 1e3   # mu = 0 has error 1

    assert diverged(1.0, 0.6) and diverged(5.0, 0.6) and diverged(10.0, 0.8)
    for c in (10.0, 20.0):
        m1, _, msg, ok = pw.run(P, h, c, 0.6, 1000)
        m2, _, _, ok2 = pw.run(P, h, c, 0.6, 1000, messages=msg)
        assert ok and ok2
        e1 = np.linalg.norm(m1 - exact) / np.linalg.norm(exact)
        e2 = np.linalg.norm(m2 - exact) / np.linalg.norm(exact)
        assert e2 < e1 < 1.0, (c, e1, e2)


def _golden_grid_search():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "pairwise_grid_search_128.txt")
    rows = [ln.split(":") for ln in open(path) if ln.strip() and not ln.startswith("#")]
    cs = [float(v) for v in rows[0][1].split()]
    table = {float(k): [None if v == "-" else float(v) for v in vals.split()] for k, vals in rows[1:]}
    return cs, table


def test_reproduces_the_papers_grid_search_on_its_synthetic_setting():
    """The paper's synthetic setting at 128^2 with 5 % of the grid observed (App. E data, the
    App. D grid search): every (c, eta) cell diverges or converges as the paper's table says,
    and among the converging cells the order of the errors is the order of the paper's RMSE
    ratios wherever those differ.  Divergence here: the error exceeds that of mu = 0 (or a
    message is not finite) within 400 iterations; the error is against the exact mean."""
    cs, table = _golden_grid_search()
    p = gabp_synth.paper_synthetic(128, 0.05, 0)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, gamma=p.gamma)
    P, h = pw.assemble(fl)
    exact = oracle.exact_mean(fl, p.nx)
    nrm = np.linalg.norm(exact)

    def error(c, eta):
        msg = None
        for _ in range(4):   # 4 x 100 iterations, stopping at the first sign of divergence
            mean, _, msg, ok = pw.run(P, h, c, eta, 100, messages=msg)
            with np.errstate(all="ignore"):
                err = np.linalg.norm(mean - exact) / nrm
            if not ok or not np.isfinite(err) or err > 1.0:
                return None
        return err

    for eta, paper in table.items():
        ours = [error(c, eta) for c in cs]
        assert [e is None for e in ours] == [v is None for v in paper], (eta, ours, paper)
        conv = [i for i, v in enumerate(paper) if v is not None]
        for i in conv:
            for j in conv:
                if paper[i] < paper[j]:
                    assert ours[i] < ours[j], (eta, cs[i], cs[j], ours[i], ours[j])


def test_upscale_copies_the_parent_edge_in_the_same_direction():
    # brute force over the fine edges: the coarse edge from the parent of the source towards
    # the same offset, or 0 where the coarse level lacks it
    fc = oracle.build_factors(3, 4, 0.3, [0.5], [1.5], [0.2], [0.1])
    ff = oracle.build_factors(6, 7, 0.15, [1.0], [3.0], [0.2], [0.1])
    Pc, _ = pw.assemble(fc)
    Pf, _ = pw.assemble(ff)
    sc, dc, _, _ = pw.edges(Pc)
    rng = np.random.default_rng(0)
    a_c, b_c = rng.standard_normal(sc.size), rng.standard_normal(sc.size)
    lookup = {(int(s), int(d)): k for k, (s, d) in enumerate(zip(sc, dc))}
    a_f, b_f = pw.upscale((a_c, b_c), Pc, 3, 4, Pf, 6, 7)
    sf, df, _, _ = pw.edges(Pf)
    for k, (s, d) in enumerate(zip(sf, df)):
        (fy, fx), (ty, tx) = divmod(int(s), 6), divmod(int(d), 6)
        py, px = min(fy // 2, 3), min(fx // 2, 2)
        qy, qx = py + ty - fy, px + tx - fx
        key = (py * 3 + px, qy * 3 + qx) if 0 <= qy < 4 and 0 <= qx < 3 else None
        want = (a_c[lookup[key]], b_c[lookup[key]]) if key in lookup else (0.0, 0.0)
        assert (a_f[k], b_f[k]) == want


def test_early_stop_rule_matches_a_step_by_step_run():
    fl = _grid_point_problem(24, 0.3, 0.1)
    P, h = pw.assemble(fl)
    t, mean, _, _, ok = pw.run_early_stop(P, h, 10.0, 0.6, 1e-2, 5000)
    assert ok and t is not None
    # independent loop: one iteration at a time, the rule of App. B by hand
    msgs = [(np.zeros(pw.edges(P)[0].size),) * 2]
    for _ in range(t):
        msgs.append(pw.run(P, h, 10.0, 0.6, 1, messages=msgs[-1])[2])
    change = [pw.message_change(msgs[i], msgs[i - 1]) for i in range(1, t + 1)]
    ref = change[1]
    first = next(i + 1 for i in range(2, t) if change[i] < 1e-2 * ref)
    assert first == t
    np.testing.assert_allclose(mean, pw.run(P, h, 10.0, 0.6, 0, messages=msgs[-1])[0], rtol=1e-14)


def test_multigrid_levels_and_fixed_point():
    p = gabp_synth.paper_synthetic(64, 0.1, 1)
    # the paper's rule: level k sees the observations on multiples of 2^k
    for k in (1, 2):
        ox, oy, _, _ = pw.level_observations(p.obs_x, p.obs_y, p.y, p.noise_var, k)
        expect = np.sum((np.mod(p.obs_x, 1 << k) == 0) & (np.mod(p.obs_y, 1 << k) == 0))
        assert ox.size == expect and np.all(ox == np.round(ox))
    # with a strict rule the levels converge, and the target reaches the exact mean
    mean, _, stop = pw.multigrid(p.nx, p.ny, p.kappa, p.gamma, p.obs_x, p.obs_y, p.y, p.noise_var,
                                 3, 10.0, 0.6, 1e-9, 20000)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, gamma=p.gamma)
    exact = oracle.exact_mean(fl, p.nx)
    assert all(t is not None for t in stop.values())
    assert np.linalg.norm(mean - exact) / np.linalg.norm(exact) < 1e-6


def test_multigrid_reference_change_readings():
    """App. B writes the rule's m_1, m_2 without a level.  Reading "level" (the library's): each
    level compares with the change between its own first two iterations.  Reading "first": every
    level compares with that change of the coarsest level.  Checked by hand: the coarsest level
    stops at the same iteration under both, and each finer level under "first" stops at the
    first iteration whose change, from the upscaled start, is below tau times the coarsest
    level's reference (a step-by-step run of the same level)."""
    p = gabp_synth.paper_synthetic(32, 0.1, 2)
    args = (p.nx, p.ny, p.kappa, p.gamma, p.obs_x, p.obs_y, p.y, p.noise_var, 2, 10.0, 0.6, 1e-3, 20000)
    _, _, stop_l = pw.multigrid(*args, reference="level")
    mean_f, _, stop_f = pw.multigrid(*args, reference="first")
    assert stop_l[1] == stop_f[1] and stop_f[0] is not None
    # by hand: the coarse level (k = 1) and its reference, then the fine level from the upscaled
    # edges, one iteration at a time
    lox, loy, ly, lv = pw.level_observations(p.obs_x, p.obs_y, p.y, p.noise_var, 1)
    nxc, nyc = -(-p.nx // 2), -(-p.ny // 2)
    flc = oracle.build_factors(nxc, nyc, p.kappa * 2, lox, loy, ly, lv, gamma=p.gamma / 4)
    Pc, hc = pw.assemble(flc)
    msgs = [(np.zeros(pw.edges(Pc)[0].size),) * 2]
    for _ in range(stop_l[1]):
        msgs.append(pw.run(Pc, hc, 10.0, 0.6, 1, messages=msgs[-1])[2])
    ref = pw.message_change(msgs[2], msgs[1])
    flf = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, gamma=p.gamma)
    Pf, hf = pw.assemble(flf)
    cur = pw.upscale(msgs[-1], Pc, nxc, nyc, Pf, p.nx, p.ny)
    t = 0
    while True:
        nxt = pw.run(Pf, hf, 10.0, 0.6, 1, messages=cur)[2]
        t += 1
        if t >= 3 and pw.message_change(nxt, cur) < 1e-3 * ref:
            break
        cur = nxt
        assert t < 20000
    assert t == stop_f[0]
    assert np.all(np.isfinite(mean_f))
