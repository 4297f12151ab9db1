"""Domain-decomposed GaBP on CPU ranks: the oracle's synchronous iteration split over the
ranks of a ``torch.distributed`` process group, with the border messages exchanged between
iterations.

TEST INFRASTRUCTURE ONLY (as the rest of ``oracle/``).  It checks the multi-device design of
the paper's Sec. 3.2.1 ("Computational Efficiency": the nodes of the graph divided into
subdomains split between compute nodes, with messages exchanged across the subdomain borders,
possibly asynchronously) on the CPU, with no GPU involved.

Partition: the grid rows are cut into ``world`` contiguous blocks.  A factor belongs to the
rank owning its anchor node: a prior cell factor (the first ``n_cells`` factors of
``build_factors``) to its cell's node, an observation factor to its base node (its smallest
variable index).  A rank updates its own factors only.  The cavity of one of its slots reads
every message into that slot's variable, so a rank needs the messages of the other ranks'
slots on the variables its factors touch (one or two grid rows across each border).  Before
an iteration the ranks exchange exactly those: rank r sends rank q the current values of
r's slots on the variables q's factors touch.

With an exchange before every iteration (``delay`` = 1), every rank computes each of its
messages from the same previous-iteration values, summed in the same slot order, as the
serial oracle does: the result is bit-identical to ``oracle.gabp``.  With ``delay`` = k the
remote messages are up to k - 1 iterations old between exchanges (the asynchronous exchange
the paper allows); the fixed point is unchanged, so a converged run reaches the same means.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import FactorList, _f64p, _i64p, _p, init_messages, lib


def row_owner(nx: int, ny: int, world: int) -> np.ndarray:
    """Rank of every node: rows split into ``world`` contiguous blocks (sizes differ by <= 1)."""
    rows = np.arange(ny)
    rank_of_row = (rows * world) // ny
    return np.repeat(rank_of_row, nx).astype(np.int64)


def factor_owner(fl: FactorList, node_rank: np.ndarray, n_cells: int) -> np.ndarray:
    """Rank of every factor: cell factors by their cell, observation factors by their base node."""
    nf = fl.nf
    anchor = np.empty(nf, np.int64)
    anchor[:n_cells] = np.arange(n_cells)
    for f in range(n_cells, nf):
        anchor[f] = fl.var[fl.ptr[f]:fl.ptr[f + 1]].min()
    return node_rank[anchor]


class Plan:
    """The static exchange plan, identical on every rank (computed from the whole graph)."""

    def __init__(self, fl: FactorList, owner: np.ndarray, world: int):
        self.world = world
        slot_factor = np.repeat(np.arange(fl.nf), np.diff(fl.ptr))
        self.slot_owner = owner[slot_factor]
        self.factors = [np.flatnonzero(owner == r).astype(np.int64) for r in range(world)]
        # variables each rank's factors touch
        touched = []
        for r in range(world):
            mask = np.zeros(fl.n, bool)
            mask[fl.var[self.slot_owner == r]] = True
            touched.append(mask)
        # send[r][q]: r's own slots on variables q's factors touch (ascending slot index)
        self.send = [[np.flatnonzero((self.slot_owner == r) & touched[q][fl.var]).astype(np.int64)
                      if q != r else np.zeros(0, np.int64) for q in range(world)] for r in range(world)]
        self.own_slots = [np.flatnonzero(self.slot_owner == r) for r in range(world)]


def _exchange(plan: Plan, rank: int, me: np.ndarray, ml: np.ndarray) -> int:
    """Send this rank's border messages and receive the others' (point to point, non-blocking
    sends and receives).  Returns the number of values received."""
    import torch
    import torch.distributed as dist
    reqs, bufs = [], []
    for q in range(plan.world):
        idx = plan.send[rank][q]
        if q != rank and idx.size:
            t = torch.from_numpy(np.stack([me[idx], ml[idx]]))
            reqs.append(dist.isend(t, q))
            bufs.append(t)
    recv = []
    for q in range(plan.world):
        idx = plan.send[q][rank]
        if q != rank and idx.size:
            t = torch.empty((2, idx.size), dtype=torch.float64)
            reqs.append(dist.irecv(t, q))
            recv.append((idx, t))
    for rq in reqs:
        rq.wait()
    got = 0
    for idx, t in recv:
        a = t.numpy()
        me[idx] = a[0]
        ml[idx] = a[1]
        got += idx.size
    return got


def gabp(fl: FactorList, nx: int, ny: int, n_cells: int, beta: float, iters: int, *, delay: int = 1,
         init: str = "cold"):
    """Run ``iters`` damped iterations split over the current process group's ranks.

    Every rank returns the same ``(mean, var, (msg_eta, msg_lam), received)``: the marginals
    and messages assembled from all ranks (each rank's own slots), and the number of message
    values this rank received over the run.  ``delay`` = iterations between exchanges."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    plan = Plan(fl, factor_owner(fl, row_owner(nx, ny, world), n_cells), world)
    me, ml = init_messages(fl, init)
    te, tl = me.copy(), ml.copy()
    fids = plan.factors[rank]
    L = lib()
    received = 0
    for t in range(iters):
        if t % delay == 0:
            received += _exchange(plan, rank, me, ml)
        rc = L.orc_iterate_factors(fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(fl.coef, _f64p),
                                   _p(fl.s, _f64p), _p(fl.r, _f64p), float(beta), int(fids.size),
                                   _p(fids, _i64p), _p(me, _f64p), _p(ml, _f64p), _p(te, _f64p), _p(tl, _f64p))
        if rc != 0:
            raise RuntimeError(f"orc_iterate_factors failed ({rc})")
        own = plan.own_slots[rank]
        me[own] = te[own]
        ml[own] = tl[own]
    # assemble: every rank contributes its own slots (others zero); the sum is exact
    out = torch.from_numpy(np.stack([np.where(plan.slot_owner == rank, me, 0.0),
                                     np.where(plan.slot_owner == rank, ml, 0.0)]))
    dist.all_reduce(out)
    ge, gl = out[0].numpy().copy(), out[1].numpy().copy()
    be = np.zeros(fl.n)
    bl = np.zeros(fl.n)
    L.orc_beliefs(fl.n, fl.nf, _p(fl.ptr, _i64p), _p(fl.var, _i64p), _p(ge, _f64p), _p(gl, _f64p),
                  _p(be, _f64p), _p(bl, _f64p))
    with np.errstate(divide="ignore", invalid="ignore"):
        return be / bl, 1.0 / bl, (ge, gl), received
