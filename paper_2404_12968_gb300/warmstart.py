"""Training and evaluation of the learned warm start.

    python -m paper_2404_12968_gb300.warmstart train --count 2000 --epochs 8 --out wsnet.npy
    python -m paper_2404_12968_gb300.warmstart eval --weights wsnet.npy
    python -m paper_2404_12968_gb300.warmstart step-time [--batch 8 --side 512 --steps 10 --warmup 3]

Training data: plain-GaBP posteriors that the library itself computes.  Problems of 512^2
nodes (kappa ~ U[0.02, 0.2], 8-32 satellite-like tracks, sigma 0.05) are solved in batches of
64 to relative residual 1e-5; each converged problem gives one sample: network input scattered
from its observations on the GPU, target = its beliefs (mean / scale, log precision).  The
network is trained on the GPU by the library's own forward and backward kernels (Adam, mean
squared error).  Evaluation: on a 2048^2 problem (kappa 0.03, 48 tracks) the time to relative
residual 1e-5 from the cold start, from the learned warm start (scatter + network inference
+ message initialisation included) and from the multigrid warm start (the paper's own
accelerator: a coarse level solved to 1e-4, upscaled; its iterations included); and the
paper's own pairwise re-weighted form (c = 20, learning rate 0.6) from zero messages, capped
at 12000 iterations.  ``step-time``: the time of one forward and backward pass (all weight
gradients) on random inputs, with the tcgen05 kernels and with the mma.sync kernels.

PyTorch only holds the samples in device memory; every computation runs in libgabp.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gabp_synth  # noqa: E402
from paper_2404_12968_gb300 import (Batch, Multigrid, Pairwise, Solver, WarmStartNet, gabp_batch_input_shape,  # noqa: E402
                                    gabp_batch_wsnet_sample, gabp_wsnet_train_step)

DAMPING = 0.3
TOL = 1e-5


def generate(count: int, side: int = 512, batch: int = 64, device: int = 0, log=print):
    """Solve `count` training problems; returns lists of device tensors (inputs, targets)."""
    import torch
    dev = torch.device("cuda", device)
    xs, ts = [], []
    t0 = time.time()
    for start in range(0, count, batch):
        probs = [gabp_synth.config_warm_train(i, side) for i in range(start, min(count, start + batch))]
        with Batch(probs, tol=TOL, check_every=20, device=device) as b:
            b.iterate(-1, DAMPING)
            for i in range(len(probs)):
                H, W, _ = gabp_batch_input_shape(b.handle, i)
                x = torch.empty((H, W, 16), dtype=torch.int16, device=dev)
                t = torch.empty((H, W, 2), dtype=torch.float32, device=dev)
                gabp_batch_wsnet_sample(b.handle, i, x, t)
                xs.append(x)
                ts.append(t)
        log(f"generated {len(xs)}/{count} samples, {time.time() - t0:.1f} s")
    return xs, ts


def train(net: WarmStartNet, xs, ts, epochs: int = 8, batch: int = 8, lr: float = 1e-3, seed: int = 0, log=print):
    H, W = int(xs[0].shape[0]), int(xs[0].shape[1])
    rng = np.random.default_rng(seed)
    steps = epochs * (len(xs) // batch)
    step = 0
    t0 = time.time()
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(xs))
        losses = []
        for s in range(0, len(order) - batch + 1, batch):
            idx = order[s:s + batch]
            # cosine decay of the learning rate
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(1, steps)))
            losses.append(gabp_wsnet_train_step(net.handle, [xs[i] for i in idx], [ts[i] for i in idx], H, W,
                                                max(lr_t, 1e-6)))
            step += 1
        hist.append(float(np.mean(losses)))
        log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.4f}, {time.time() - t0:.1f} s")
    return hist


MG_LEVELS = 2      # multigrid: one coarse level (the best of 2..7 levels at 2048^2)
MG_TOL = 1e-4      # relative residual the coarse level is solved to
PW_C, PW_ETA = 20.0, 0.6   # the paper's pairwise form (its c = 10 diverges on this problem)
PW_CHECK, PW_MAX = 500, 12000


def pairwise_to_tol(solver: Solver, tol: float = TOL, means: dict | None = None):
    """The paper's pairwise re-weighted form from zero messages: residual checked every
    PW_CHECK iterations, at most PW_MAX; (seconds, iterations, residual).  With ``means`` given,
    the final marginal means are stored under "pairwise"."""
    with Pairwise(solver) as pw:
        pw.iterate(2, PW_C, PW_ETA)    # warm-up launch
        pw.reset()
        t0 = time.perf_counter()
        its, r = 0, float("nan")
        while its < PW_MAX:
            pw.iterate(PW_CHECK, PW_C, PW_ETA)
            its += PW_CHECK
            r = pw.residual()
            if not r > tol:
                break
        dt = time.perf_counter() - t0
        if means is not None:
            means["pairwise"] = pw.marginals(want_var=False)[0]
        return dt, its, r


def time_to_tol(solver: Solver, net: WarmStartNet | None, tol: float = TOL, check_every: int = 10, mg=None):
    """Seconds (wall, synchronous calls) and iterations from a fresh start to `tol`: cold, after
    the learned warm start (`net`), or after the multigrid warm start (`mg`, coarse levels
    included in the time and counted separately)."""
    solver.reset()
    coarse = 0
    t0 = time.perf_counter()
    if net is not None:
        solver.learned_warm_start(net)
    if mg is not None:
        coarse = sum(mg.warm_start(DAMPING, MG_TOL, 100000)["iterations"])
    solver.iterate(-1, DAMPING)
    dt = time.perf_counter() - t0
    st = solver.stats()
    return dt, int(st["iterations"]), float(st["last_residual"]), coarse


def evaluate(net: WarmStartNet, problem=None, device: int = 0, repeats: int = 3, means: dict | None = None):
    """Time to TOL from the cold start, the learned warm start, the multigrid warm start and the
    pairwise form.  With ``means`` given, the final marginal means of each ("cold", "warm",
    "multigrid", "pairwise") are stored there (read after the timed runs)."""
    p = problem if problem is not None else gabp_synth.config_warm_eval(0)
    with Solver(p, precision="fp32", tol=TOL, check_every=10, max_iters=400000, device=device) as s:
        with Multigrid(s, MG_LEVELS) as mg:      # the coarse problem is set up once, like the solver
            time_to_tol(s, None)                 # warm-up (graph capture, first launches)
            time_to_tol(s, net)
            time_to_tol(s, None, mg=mg)
            cold = [time_to_tol(s, None) for _ in range(repeats)]
            if means is not None:
                means["cold"] = s.marginals(want_var=False)[0]
            warm = [time_to_tol(s, net) for _ in range(repeats)]
            if means is not None:
                means["warm"] = s.marginals(want_var=False)[0]
            mgr = [time_to_tol(s, None, mg=mg) for _ in range(repeats)]
            if means is not None:
                means["multigrid"] = s.marginals(want_var=False)[0]
        pw_s, pw_its, pw_res = pairwise_to_tol(s, means=means)
    best = lambda r: min(r, key=lambda z: z[0])  # noqa: E731
    c, w, g = best(cold), best(warm), best(mgr)
    return {"grid": [p.nx, p.ny], "kappa": p.kappa, "m": p.m, "tol": TOL, "damping": DAMPING,
            "cold_s": c[0], "cold_iters": c[1], "warm_s": w[0], "warm_iters": w[1],
            "speedup": c[0] / w[0], "cold_residual": c[2], "warm_residual": w[2],
            "multigrid_s": g[0], "multigrid_iters": g[1], "multigrid_coarse_iters": g[3],
            "multigrid_levels": MG_LEVELS, "multigrid_coarse_tol": MG_TOL, "multigrid_speedup": c[0] / g[0],
            "multigrid_residual": g[2],
            "pairwise_c": PW_C, "pairwise_learning_rate": PW_ETA, "pairwise_s": pw_s, "pairwise_iters": pw_its,
            "pairwise_residual": pw_res, "pairwise_reached_tol": bool(pw_res <= TOL)}


def step_time(batch: int, side: int, steps: int = 10, warmup: int = 3) -> dict:
    """Milliseconds per forward and backward pass (every layer's gradients) on random inputs
    of ``batch`` x side^2, for each set of convolution kernels (CUDA events on the default
    stream around ``steps`` passes after ``warmup``)."""
    import torch
    from paper_2404_12968_gb300 import (GABP_WSNET_MMA_SYNC, GABP_WSNET_TCGEN05, gabp_wsnet_gradients,
                                        gabp_wsnet_param_count, gabp_wsnet_set_kernels)
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev).manual_seed(0)
    xs = [torch.randn(side, side, 16, device=dev, generator=gen).to(torch.bfloat16).view(torch.int16)
          for _ in range(batch)]
    ts = [torch.randn(side, side, 2, device=dev, generator=gen) for _ in range(batch)]
    net = WarmStartNet(seed=1, device=0)
    g = np.empty(gabp_wsnet_param_count(net.handle), np.float32)
    out = {"batch": batch, "side": side}
    try:
        for name, k in (("tcgen05", GABP_WSNET_TCGEN05), ("mma_sync", GABP_WSNET_MMA_SYNC)):
            gabp_wsnet_set_kernels(net.handle, k)
            for _ in range(warmup):
                gabp_wsnet_gradients(net.handle, xs, ts, side, side, g)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                gabp_wsnet_gradients(net.handle, xs, ts, side, side, g)
            torch.cuda.synchronize()
            out[f"{name}_ms"] = (time.perf_counter() - t0) / steps * 1e3
            out[f"{name}_grad_norm"] = float(np.linalg.norm(g))
    finally:
        net.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["train", "eval", "step-time"])
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--side", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="wsnet.npy")
    ap.add_argument("--weights", default=None)
    ap.add_argument("--eval-side", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=10, help="step-time: timed passes per kernel set")
    ap.add_argument("--warmup", type=int, default=3, help="step-time: untimed passes first")
    args = ap.parse_args()
    if args.mode == "step-time":
        print(json.dumps(step_time(args.batch, args.side, args.steps, args.warmup)), flush=True)
        return
    net = WarmStartNet(seed=args.seed, device=0)
    report = {}
    if args.mode == "train":
        t0 = time.time()
        xs, ts = generate(args.count, args.side)
        report["generate_s"] = time.time() - t0
        t0 = time.time()
        report["loss_per_epoch"] = train(net, xs, ts, args.epochs, args.batch, args.lr, args.seed)
        report["train_s"] = time.time() - t0
        net.save(args.out)
        del xs, ts
    else:
        net.load(args.weights)
    report["eval"] = evaluate(net, gabp_synth.config_warm_eval(0, args.eval_side))
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
