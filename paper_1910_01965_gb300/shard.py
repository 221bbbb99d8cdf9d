"""Sharding a scan over ranks: each rank takes a contiguous slice of the
flat grid index, computes it with no exchange, and the slices are gathered
on the host (or not at all).

Every (grid point, trial) unit is independent and its random stream is keyed
by the global flat index, so a slice reproduces the same points of a
whole-grid scan bit for bit; the only communication is the host-side gather
of disjoint slices and the timing reduction of the benchmark.  This is the
paper's batches-to-GPUs scheme (Sec. 2) without a task scheduler.
"""
from __future__ import annotations

import time
from typing import Callable, Dict, Tuple

import numpy as np


def shard_range(P: int, rank: int, world: int) -> Tuple[int, int]:
    """(first_index, count) of rank's contiguous slice of [0, P); the first
    P mod world ranks take one extra point."""
    if world < 1 or not 0 <= rank < world or P < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(P, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    return dist


def _device():
    import torch
    dist = _dist()
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(value: float) -> float:
    """Largest `value` over all ranks (1 rank: the value itself)."""
    dist = _dist()
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    dist = _dist()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def gather_slices(local: np.ndarray, P: int) -> np.ndarray:
    """Host-side gather of every rank's slice into the whole grid (all ranks
    receive it).  `local` holds this rank's shard_range slice: one value per
    point, or one row per point (e.g. the per-trial sums)."""
    local = np.asarray(local)
    dist = _dist()
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    world, rank = dist.get_world_size(), dist.get_rank()
    parts = [None] * world
    dist.all_gather_object(parts, (rank, local))
    out = np.empty((P,) + local.shape[1:], dtype=local.dtype)
    for r, arr in parts:
        first, count = shard_range(P, r, world)
        out[first:first + count] = arr
    return out


def sharded_scan(P: int, scan_slice: Callable[[int, int], Dict[str, np.ndarray]]):
    """One sharded pass over a grid of P points: this rank runs
    ``scan_slice(first, count)`` on its shard_range slice between two
    barriers, the wall time is reduced to the slowest rank, and every output
    array the function returns (a value or a row per point of the slice) is
    gathered into the whole grid.  Returns (gathered arrays, slowest rank's
    seconds)."""
    dist = _dist()
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size() if on else 1
    rank = dist.get_rank() if on else 0
    first, count = shard_range(P, rank, world)
    barrier()
    t0 = time.perf_counter()
    local = scan_slice(first, count)
    barrier()
    slowest = max_over_ranks(time.perf_counter() - t0)
    return {k: gather_slices(v, P) for k, v in local.items()}, slowest
