"""Write the stored exact posterior means of the full-size workloads (sampled nodes).

    python tests/golden/make_exact_means.py [name ...]

The full-size grids (4096^2 and the 2048^2 warm-start evaluation) are too large for the
oracle to solve inside a GPU test or the benchmark's bounded run, so their exact posterior
means A^-1 b are computed once here, by the oracle alone (``oracle.exact.exact_mean_pcg``,
FP64 preconditioned conjugate gradients to ||b - A x|| / ||b|| <= 4e-15 where the iteration
reaches it, else 1e-13), and stored at a
seeded uniform sample of nodes together with the full field's L2 norm.  The inputs come from
the shared seeded generator ``gabp_synth``; each file records checksums of them so that a
reader can tell the generator still produces the same problem.  Nothing here touches the CUDA
library.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gabp_synth  # noqa: E402

SAMPLES = 4096
BATCH_INSTANCES = (0, 5, 11, 23, 37, 42, 50, 63)


def roofline_scaled(side: int, seed: int = 0):
    """The 4096^2 workload's generator at another size, observation counts scaled with the area."""
    f = (side / 4096.0) ** 2
    return gabp_synth.make_problem(side, side, 0.02, seed, n_uniform=int(200_000 * f), n_tracks=96,
                                   per_track=max(1, int(round(1_200_000 * f / 96))), sigma=(0.02, 0.1))


def workloads():
    """name -> (problem maker, description, alpha)."""
    out = {
        "roofline_4096": (lambda: gabp_synth.config_roofline_4096(0),
                          "4096x4096, kappa 0.02, 96 tracks (1.2M samples) + 200k uniform points, sigma ~ U[0.02, 0.1], seed 0", 2),
        "warm_eval_2048": (lambda: gabp_synth.config_warm_eval(0),
                           "2048x2048, kappa 0.03, 48 tracks, sigma 0.05 (the warm-start evaluation problem), seed 0", 2),
        "tracks_1024": (lambda: gabp_synth.config_tracks_1024(0),
                        "1024x1024, kappa 0.05, 24 tracks (~40k samples), sigma 0.05, seed 0", 2),
        "roofline_512_alpha4": (lambda: roofline_scaled(512),
                                "the 4096^2 workload's generator at 512x512 (observations scaled with the area), "
                                "alpha = 4 prior (cell factors = rows of L^2), seed 0", 4),
    }
    for i in BATCH_INSTANCES:
        out[f"batch_{i:02d}"] = ((lambda i=i: gabp_synth.config_batch(seed=0)[i]),
                                 f"instance {i} of the 64-instance batch (seed 0)", 2)
    return out


def path_for(name: str) -> str:
    return os.path.join(HERE, f"exact_mean_{name}.txt")


def input_checksums(p) -> dict:
    return {"sum_obs_x": float(np.sum(p.obs_x)), "sum_obs_y": float(np.sum(p.obs_y)),
            "sum_y": float(np.sum(p.y)), "sum_noise_var": float(np.sum(p.noise_var))}


def sample_indices(n: int, name: str) -> np.ndarray:
    seed = sum(ord(c) for c in name) * 7919
    k = min(SAMPLES, n)
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


def write(name: str, verbose: bool = True) -> str:
    import oracle
    from oracle import exact
    make, desc, alpha = workloads()[name]
    p = make()
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var, p.gamma, alpha)
    t = time.time()
    # the solve's own error is about (condition number) x (relative residual): at 1024^2 the
    # solutions at 1e-13 and 3e-15 differ by 2.4e-10, so the stored means are solved to 4e-15
    # where the iteration gets there (1e-13 otherwise), well below the 1e-10 of the FP64 bar
    try:
        x, info = exact.exact_mean_pcg(fl, p.nx, p.ny, tol=4e-15, maxit=20000, verbose=verbose)
    except RuntimeError:
        x, info = exact.exact_mean_pcg(fl, p.nx, p.ny, tol=1e-13, maxit=20000, verbose=verbose)
    dt = time.time() - t
    idx = sample_indices(p.n, name)
    cs = input_checksums(p)
    lines = [
        f"# Exact posterior mean A^-1 b at {len(idx)} sampled nodes: {desc}.",
        "# Written by tests/golden/make_exact_means.py with the oracle alone (FP64 PCG with a",
        f"# multigrid preconditioner, run to ||b - A x|| / ||b|| = {info['rel_residual']:.2e}).",
        f"# nx {p.nx}", f"# ny {p.ny}", f"# kappa {p.kappa!r}", f"# gamma {p.gamma!r}", f"# alpha {alpha}",
        f"# m {p.m}",
        *[f"# {k} {v!r}" for k, v in cs.items()],
        f"# norm_full {float(np.linalg.norm(x))!r}",
        f"# pcg_iterations {info['iterations']}",
        f"# rel_residual {info['rel_residual']!r}",
        f"# solve_seconds {dt:.1f}",
        "# node_index exact_mean",
    ]
    lines += [f"{int(i)} {float(x[i])!r}" for i in idx]
    with open(path_for(name), "w") as f:
        f.write("\n".join(lines) + "\n")
    if verbose:
        print(f"{name}: {info} in {dt:.1f} s", flush=True)
    return path_for(name)


def load(name: str) -> dict:
    """The stored sample: {'index', 'mean', and every header key}."""
    meta = {}
    idx, val = [], []
    with open(path_for(name)) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) == 2:
                    try:
                        meta[parts[0]] = float(parts[1])
                    except ValueError:
                        pass
                continue
            a, b = line.split()
            idx.append(int(a))
            val.append(float(b))
    meta["index"] = np.asarray(idx, np.int64)
    meta["mean"] = np.asarray(val)
    return meta


if __name__ == "__main__":
    names = sys.argv[1:] or list(workloads())
    for nm in names:
        write(nm)
