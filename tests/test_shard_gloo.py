"""The multi-rank path on CPU: world_size 2 over gloo.

Each rank evaluates its contiguous slice of the grid (here with the oracle,
which stands in for the rank's GPU), the slices are gathered on the host, and
the result equals the whole-grid scan; the benchmark's max-over-ranks timing
reduction and barrier run through the same process group.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1910_01965_gb300 import shard


def test_shard_range_partitions_the_grid():
    for P in [0, 1, 7, 100, 10 ** 6 + 3]:
        for world in [1, 2, 3, 8]:
            spans = [shard.shard_range(P, r, world) for r in range(world)]
            assert sum(c for f, c in spans) == P
            pos = 0
            for f, c in spans:
                assert f == pos
                pos += c
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        from paper_1910_01965_gb300 import workloads as wl
        spec = wl.scan_cosprod_100(samples=1 << 10, trials=3)
        first, count = shard.shard_range(spec.P, rank, world)
        pts = np.arange(first, first + count, dtype=np.int64)
        res = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                           spec.lengths, spec.values, spec.samples,
                                           spec.trials, spec.seed, pts, nthreads=1)
        shard.barrier()
        full = shard.gather_slices(res["mean"], spec.P)
        slowest = shard.max_over_ranks(float(rank + 1))
        if rank == 0:
            q.put((full, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_shard_gather_and_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full, slowest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from oracle import oracle
    from paper_1910_01965_gb300 import workloads as wl
    spec = wl.scan_cosprod_100(samples=1 << 10, trials=3)
    whole = oracle.default().scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                  spec.values, spec.samples, spec.trials, spec.seed)
    assert np.array_equal(full, whole["mean"])
    assert slowest == 2.0


def _worker_sharded(rank, world, port, q):
    """The benchmark's sharded pass (shard.sharded_scan): slices, barriers,
    slowest-rank time, gather of per-point values and per-trial rows."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import time
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        from paper_1910_01965_gb300 import workloads as wl
        spec = wl.scan_gauss_1e6(samples=1 << 8, trials=2)
        spec.lists[0] = spec.lists[0][:3]          # 3 x 100 x 100 x 1 = 30,000 points
        spec.lists[1] = spec.lists[1][:7]          # ... cut to 2,100 points

        def scan_slice(first, count):
            if rank == 1:
                time.sleep(0.3)                    # the slower rank sets the time
            pts = np.arange(first, first + count, dtype=np.int64)
            res = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                               spec.lengths, spec.values, spec.samples,
                                               spec.trials, spec.seed, pts, nthreads=1,
                                               want_sums=True)
            return {"mean": res["mean"], "s1": res["s1"]}
        full, slowest = shard.sharded_scan(spec.P, scan_slice)
        if rank == 0:
            q.put((full["mean"], full["s1"], slowest, spec.P))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_sharded_scan_helper():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_sharded, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    mean, s1, slowest, P = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from oracle import oracle
    from paper_1910_01965_gb300 import workloads as wl
    spec = wl.scan_gauss_1e6(samples=1 << 8, trials=2)
    spec.lists[0] = spec.lists[0][:3]
    spec.lists[1] = spec.lists[1][:7]
    whole = oracle.default().scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                  spec.values, spec.samples, spec.trials, spec.seed,
                                  want_sums=True)
    assert P == spec.P and mean.shape == (P,) and s1.shape == (P, 2)
    assert np.array_equal(mean, whole["mean"]) and np.array_equal(s1, whole["s1"])
    assert slowest >= 0.3
