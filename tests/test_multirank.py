"""Multi-rank host logic on CPU (gloo, world size 2): the cell decomposition and
two-cell halo exchange reproduce the single-domain transport, and the
benchmark's max-over-ranks timing rule."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import qbe_oracle as O
from paper_1408_1782_gb300 import decomp, inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, kind, Nx, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = O.Params(N=8)
        W = inputs.synthetic_w(8, Nx, seed=5) + 0.02 * np.random.default_rng(1).normal(size=(Nx, 4, 8, 8))
        fd = (1.0, 0.2, -0.3, np.eye(2))
        bc = O.Boundary(kind, fd, fd, alpha=0.6)
        lo, hi = decomp.block_range(rank, world, Nx)
        block = W[lo:hi]
        dx, tau = 1.0 / Nx, 0.8 / Nx / p.L
        for _ in range(3):
            left, right = decomp.halo_exchange(torch.from_numpy(block), periodic=(kind == "periodic"))
            wall = O._ghosts(block, p, bc) if kind != "periodic" else None
            gl = left.numpy() if left is not None else wall[:2]
            gr = right.numpy() if right is not None else wall[-2:]
            block = O.limiter_update(np.concatenate([gl, block, gr]), tau, dx, p)
        t = decomp.max_over_ranks(float(rank + 1))
        gathered = [None] * world
        dist.all_gather_object(gathered, (lo, hi, block, t))
        if rank == 0:
            full = np.empty_like(W)
            for (a, b, blk, tt) in gathered:
                full[a:b] = blk
            ref = W
            for _ in range(3):
                ref = O.advect_substep(ref, tau, dx, p, bc)
            out.put((np.abs(full - ref).max(), [g[3] for g in gathered]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind,Nx", [("periodic", 9), ("dirichlet", 7), ("maxwell", 8)])
def test_two_rank_halo_exchange_matches_single_domain(kind, Nx):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, Nx, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    err, times = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert err == 0.0
    assert times == [2.0, 2.0]


def test_block_ranges_cover_the_cells():
    for Nx, world in ((9, 2), (128, 8), (7, 3)):
        spans = [decomp.block_range(r, world, Nx) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == Nx
        assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
        assert all(b - a >= 2 for a, b in spans)
    with pytest.raises(ValueError):
        decomp.block_range(0, 4, 7)
