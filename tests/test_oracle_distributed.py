"""The domain-decomposed oracle (Sec. 3.2.1: subdomains on separate compute nodes, border
messages exchanged) on CPU gloo ranks: with an exchange before every iteration it is
bit-identical to the serial oracle; with a delayed exchange it converges to the same means."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NX, NY, KAPPA, SEED = 40, 33, 0.3, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    sys.path.insert(0, ROOT)
    import gabp_synth
    import oracle
    p = gabp_synth.make_problem(NX, NY, KAPPA, SEED, n_tracks=2, per_track=NX, n_uniform=150)
    fl = oracle.build_factors(p.nx, p.ny, p.kappa, p.obs_x, p.obs_y, p.y, p.noise_var)
    return p, fl


def _rank_main(rank, world, port, runs, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from oracle import distributed
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, fl = _problem()
        out = []
        for beta, iters, delay in runs:
            mean, var, msg, got = distributed.gabp(fl, p.nx, p.ny, p.n, beta, iters, delay=delay)
            out.append((mean, var, msg, got))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _run(world, runs):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, runs, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_synchronous_exchange_is_bit_identical_to_the_serial_run(world):
    import oracle
    p, fl = _problem()
    beta, iters = 0.5, 37
    mean_s, var_s, (me_s, ml_s) = oracle.gabp(fl, beta, iters)
    res = _run(world, [(beta, iters, 1)])
    for rank in range(world):
        mean, var, (me, ml), got = res[rank][0]
        assert np.array_equal(me, me_s) and np.array_equal(ml, ml_s), rank
        assert np.array_equal(mean, mean_s) and np.array_equal(var, var_s), rank
        assert got > 0, rank
    # only border messages travel: far fewer than the rank's whole message set
    assert max(res[r][0][3] for r in range(world)) < 0.25 * iters * fl.ne


def test_partition_covers_every_factor_once_and_exchanges_only_border_rows():
    import oracle
    from oracle import distributed
    p, fl = _problem()
    world = 3
    node_rank = distributed.row_owner(p.nx, p.ny, world)
    owner = distributed.factor_owner(fl, node_rank, p.n)
    plan = distributed.Plan(fl, owner, world)
    allf = np.sort(np.concatenate(plan.factors))
    assert np.array_equal(allf, np.arange(fl.nf))
    rows = np.arange(fl.n) // p.nx
    for r in range(world):
        for q in range(world):
            idx = plan.send[r][q]
            if not idx.size:
                continue
            assert abs(r - q) == 1   # only neighbouring row blocks share variables
            # the variables of the exchanged slots lie within two rows of the border
            border = min(np.flatnonzero(node_rank.reshape(p.ny, p.nx)[:, 0] == max(r, q)))
            assert np.all(np.abs(rows[fl.var[idx]] - border) <= 2)


def test_delayed_exchange_converges_to_the_same_means():
    import oracle
    p, fl = _problem()
    exact = oracle.exact_mean(fl, p.nx)
    beta, iters = 0.5, 400
    res = _run(2, [(beta, iters, 1), (beta, iters, 4)])
    sync_mean = res[0][0][0]
    delayed_mean = res[0][1][0]
    nrm = np.linalg.norm(exact)
    assert np.linalg.norm(sync_mean - exact) / nrm < 1e-9
    assert np.linalg.norm(delayed_mean - exact) / nrm < 1e-9
    # the delayed run exchanged a quarter as often
    assert res[0][1][3] * 4 == res[0][0][3]
