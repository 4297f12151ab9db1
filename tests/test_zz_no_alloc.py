"""The allocation-free residual entry point (gabp_residual_noalloc) against gabp_residual.

gabp_residual_noalloc serves callers that cannot allocate device memory through the library
(for example when another allocator already holds the device memory): it takes every input and
the output from the caller and keeps its scratch in a static device array.  This file is named
to be collected last, so that a run stopping at the first failure has run every other test
first; it also passes when run alone in a fresh process."""
import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built

pytestmark = pytest.mark.gpu


def _sorted_device_obs(p, torch, dev):
    j0 = np.minimum(np.floor(p.obs_x), p.nx - 2)
    i0 = np.minimum(np.floor(p.obs_y), p.ny - 2)
    order = np.argsort(i0 * p.nx + j0, kind="stable")
    xy = np.ascontiguousarray(np.stack([p.obs_x[order], p.obs_y[order]], axis=1).reshape(-1))
    return (torch.tensor(xy, dtype=torch.float64, device=dev),
            torch.tensor(p.y[order], dtype=torch.float64, device=dev),
            torch.tensor(p.noise_var[order], dtype=torch.float64, device=dev))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_residual_matches_context_residual(precision):
    torch = pytest.importorskip("torch")
    ensure_built()
    from paper_2404_12968_gb300 import Solver, gabp_residual_noalloc

    dev = torch.device("cuda", 0)
    p = gabp_synth.make_problem(203, 151, 0.1, 3, n_uniform=2000, n_tracks=3, per_track=150,
                                sigma=(0.02, 0.1))
    xy, yv, nv = _sorted_device_obs(p, torch, dev)
    mean = torch.empty(p.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with Solver(p, precision=precision, gamma=1.3) as s:
        for its in (40, 25):   # two calls in a row, on two different means
            s.iterate(its, 0.3)
            s.marginals(out_mean=mean, want_var=False)
            r_ref = s.residual()
            r = gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, mean, gamma=1.3, stream=stream)
            assert r == pytest.approx(r_ref, rel=1e-10, abs=0)


def test_noalloc_residual_rejects_bad_input():
    torch = pytest.importorskip("torch")
    ensure_built()
    from paper_2404_12968_gb300 import GabpError, gabp_residual_noalloc

    dev = torch.device("cuda", 0)
    p = gabp_synth.make_problem(40, 30, 0.2, 1, n_uniform=100)
    xy, yv, nv = _sorted_device_obs(p, torch, dev)
    mean = torch.zeros(p.n, dtype=torch.float64, device=dev)
    # larger than the static scratch: rejected before any GPU work
    big = torch.zeros(2048 * 2048, dtype=torch.float64, device=dev)
    with pytest.raises(GabpError, match="too large"):
        gabp_residual_noalloc(2048, 2048, 0.1, xy, yv, nv, big)
    del big
    # observations not sorted by base cell
    with pytest.raises(GabpError, match="sorted"):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy.view(-1, 2).flip(0).reshape(-1).contiguous(),
                              yv.flip(0).contiguous(), nv.flip(0).contiguous(), mean)
    # still usable afterwards
    r = gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, mean)
    assert r == pytest.approx(1.0)


def test_noalloc_residual_reports_out_of_grid_and_bad_variance_then_recovers():
    """Device-side checks: an observation past the last column, a zero noise variance (each
    reported as such even when the order is also broken), then a valid call."""
    torch = pytest.importorskip("torch")
    ensure_built()
    from paper_2404_12968_gb300 import GabpError, gabp_residual_noalloc

    dev = torch.device("cuda", 0)
    p = gabp_synth.make_problem(40, 30, 0.2, 2, n_uniform=100)
    xy, yv, nv = _sorted_device_obs(p, torch, dev)
    mean = torch.zeros(p.n, dtype=torch.float64, device=dev)
    bad_xy = xy.clone()
    bad_xy[2 * (p.m - 1)] = p.nx - 1 + 0.5          # last observation past the last column
    with pytest.raises(GabpError, match="outside the grid"):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, bad_xy, yv, nv, mean)
    bad_nv = nv.clone()
    bad_nv[5] = 0.0
    with pytest.raises(GabpError, match="non-positive variance"):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, bad_nv, mean)
    # both an unsorted order and a bad variance: the variance is what is reported
    rev = lambda t, w: t.view(-1, w).flip(0).reshape(-1).contiguous()   # noqa: E731
    with pytest.raises(GabpError, match="non-positive variance"):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, rev(xy, 2), rev(yv, 1), rev(bad_nv, 1), mean)
    assert gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, mean) == pytest.approx(1.0)


def test_noalloc_residual_without_observations_matches_context():
    """m = 0 skips the observation kernel and the corner loops: compared with the residual of a
    context without observations (b = 0, so both return ||A mu||)."""
    torch = pytest.importorskip("torch")
    ensure_built()
    from paper_2404_12968_gb300 import Solver, gabp_residual_noalloc

    dev = torch.device("cuda", 0)
    p = gabp_synth.make_problem(37, 29, 0.3, 4, n_uniform=0)
    rng = np.random.default_rng(5)
    mu0 = rng.standard_normal(p.n)
    empty = torch.zeros(0, dtype=torch.float64, device=dev)
    with Solver(p, precision="fp64") as s:
        s.warm_start(mu0, np.full(p.n, 2.0))
        r_ref = s.residual()
        mean = torch.tensor(s.marginals(want_var=False)[0], dtype=torch.float64, device=dev)
    r = gabp_residual_noalloc(p.nx, p.ny, p.kappa, empty, empty, empty, mean)
    assert r == pytest.approx(r_ref, rel=1e-12) and r > 0.0


def test_noalloc_wrapper_and_entry_point_refuse_unusable_arrays():
    """The binding refuses host arrays, other dtypes and wrong lengths before calling the
    library; the entry point itself refuses a host pointer (cudaPointerGetAttributes)."""
    torch = pytest.importorskip("torch")
    ensure_built()
    import ctypes
    from paper_2404_12968_gb300 import GABP_ERR_ARG, _lib, gabp_residual_noalloc

    dev = torch.device("cuda", 0)
    p = gabp_synth.make_problem(24, 20, 0.2, 6, n_uniform=30)
    xy, yv, nv = _sorted_device_obs(p, torch, dev)
    mean = torch.zeros(p.n, dtype=torch.float64, device=dev)
    with pytest.raises(TypeError):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, np.zeros(p.n))
    with pytest.raises(ValueError):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, mean.float())
    with pytest.raises(ValueError):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, mean[:-1])
    with pytest.raises(ValueError):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy[:-2], yv, nv, mean)
    host_mean = np.zeros(p.n)
    out = ctypes.c_double()
    L = _lib.load()
    rc = L.gabp_residual_noalloc(_lib.gabp_grid(p.nx, p.ny, 1.0), float(p.kappa), 1.0, p.m, xy.data_ptr(),
                                 yv.data_ptr(), nv.data_ptr(), host_mean.ctypes.data, ctypes.byref(out), None)
    assert rc == GABP_ERR_ARG
    assert b"device memory" in L.gabp_residual_noalloc_error()
    assert gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, mean) == pytest.approx(1.0)
