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
    with pytest.raises(GabpError, match="too large"):
        gabp_residual_noalloc(2048, 2048, 0.1, xy, yv, nv, mean)
    # observations not sorted by base cell
    with pytest.raises(GabpError, match="sorted"):
        gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy.view(-1, 2).flip(0).reshape(-1).contiguous(),
                              yv.flip(0).contiguous(), nv.flip(0).contiguous(), mean)
    # still usable afterwards
    r = gabp_residual_noalloc(p.nx, p.ny, p.kappa, xy, yv, nv, mean)
    assert r == pytest.approx(1.0)
