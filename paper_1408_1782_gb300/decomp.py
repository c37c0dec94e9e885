"""Spatial decomposition of the cells across ranks (paper Sec. 4: each process
owns adjacent finite volumes; the transport step needs two neighbours on each
side, so blocks hold at least two cells and exchange a two-cell halo).

Host-side logic only, written against torch.distributed point-to-point calls
so that the same code drives gloo (CPU) and NCCL (GPU) process groups.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

HALO = 2


def block_range(rank: int, world: int, Nx: int):
    """Contiguous block [lo, hi) of cells owned by `rank`; sizes differ by at most one."""
    if world * HALO > Nx:
        raise ValueError(f"{Nx} cells cannot give every one of {world} ranks at least {HALO} cells")
    base, extra = divmod(Nx, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def halo_exchange(block: torch.Tensor, periodic: bool, group=None):
    """Exchange the two outermost cells with the neighbouring ranks.

    block: [n_local, ...] cells of this rank (contiguous).  Returns (left, right):
    the two cells to the left of the block and the two to its right, or None at
    a physical wall (non-periodic ends), where the boundary condition supplies
    the ghosts.
    """
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    left_nb = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    right_nb = rank + 1 if rank < world - 1 else (0 if periodic else None)
    first = block[:HALO].contiguous()
    last = block[-HALO:].contiguous()
    left = torch.empty_like(first) if left_nb is not None else None
    right = torch.empty_like(last) if right_nb is not None else None
    # tag 0: a block's first cells travelling left; tag 1: its last cells travelling right
    # (with two ranks and periodic ends both neighbours are the same rank)
    ops = []
    if left_nb is not None:
        ops.append(dist.P2POp(dist.isend, first, left_nb, group, tag=0))
        ops.append(dist.P2POp(dist.irecv, left, left_nb, group, tag=1))
    if right_nb is not None:
        ops.append(dist.P2POp(dist.isend, last, right_nb, group, tag=1))
        ops.append(dist.P2POp(dist.irecv, right, right_nb, group, tag=0))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return left, right


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of a per-rank scalar (the benchmark's timing rule)."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
