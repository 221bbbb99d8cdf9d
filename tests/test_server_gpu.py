"""The serving loop (zmc_server.h): continuous batching, chunked streaming,
cancellation, host-side failure injection, bounded waits.

Every served result must equal the same scan run alone with the same tile
configuration bit for bit: a request's tiles depend only on the request, and
each tile computes the same sums whatever else shares the step.
"""
import threading
import time

import numpy as np
import pytest

import parity
from oracle import oracle
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc
    zmc.load()
    return zmc


def _solo(z, spec, prec, o):
    res, so = z.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                     spec.samples, spec.trials, spec.seed, precision=prec,
                     tiles=(o.tile_lanes, o.tile_splits, 256))
    return res


def _mix(n=40, seed=5):
    rng = np.random.default_rng(seed)
    specs = wl.batch_uneven_256(count=n, seed=seed)
    out = []
    for s in specs:  # keep the test short: cap grids and samples
        s.samples = int(min(s.samples, 1 << 14))
        s.lists = [v[:min(len(v), 30)] for v in s.lists]
        out.append((s, int(rng.choice([0, 1, 2], p=[0.1, 0.2, 0.7]))))
    return out


def test_served_mix_equals_solo_runs(z):
    srv = z.Server(1 << 30, max_active=16, step_ms=2.0)
    mix = _mix()
    tickets = []

    def submitter():
        rng = np.random.default_rng(1)
        for spec, prec in mix:
            time.sleep(float(rng.exponential(0.002)))
            tickets.append((srv.submit(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                       spec.lengths, spec.values, spec.samples, spec.trials,
                                       spec.seed, prec), spec, prec))

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    try:
        for t, spec, prec in tickets:
            assert srv.wait(t, 60000) == z.ZMC_OK
        st = srv.stats()
        assert st.completed == len(mix) and st.failed == 0 and st.steps >= 2
        for t, spec, prec in tickets:
            res, o = srv.result(t)
            solo = _solo(z, spec, prec, o)
            assert np.array_equal(res["mean"], solo["mean"]), spec.name
            assert np.array_equal(res["err"], solo["err"]), spec.name
            assert o.total_ms > 0
        # and the oracle agrees with a few of them
        O = oracle.default()
        for t, spec, prec in tickets[:5]:
            res, o = srv.result(t)
            ref = O.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                         spec.values, spec.samples, spec.trials, spec.seed, want_sums=True)
            V = float(np.prod(spec.hi - spec.lo))
            parity.check(res, ref, V, spec.samples, prec, spec.name + " served")
    finally:
        srv.close()


def test_chunked_streaming_of_a_large_grid(z):
    # 2^14 unit-splits per chunk: this grid (P = 60000, T = 3) streams in chunks
    srv = z.Server(1 << 30, chunk_units=1 << 14, step_ms=1.0)
    spec = wl.ScanSpec("big", wl.G_COSPROD, 3, np.zeros(3), np.ones(3),
                       [np.linspace(0.5, 5, 40), np.linspace(0.5, 5, 50),
                        np.linspace(0.5, 5, 30)], 1000, 3, 77)
    try:
        t = srv.submit(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                       spec.samples, spec.trials, spec.seed, 2, want_sums=True)
        small = srv.submit(1, 2, [0, 0], [1, 1], [5, 5], np.linspace(0.5, 5, 10), 512, 2, 3)
        assert srv.wait(t, 120000) == z.ZMC_OK and srv.wait(small, 60000) == z.ZMC_OK
        res, o = srv.result(t)
        solo = _solo(z, spec, 2, o)
        assert np.array_equal(res["mean"], solo["mean"])
        assert srv.stats().steps > 3
    finally:
        srv.close()


def test_many_chunks_of_two_grids_interleaved(z):
    # Small chunks and short steps: each request's chunks finish in consecutive
    # steps, so both output buffers are reused many times while earlier chunks
    # are still being copied to the host.  Every output equals the solo run.
    srv = z.Server(1 << 30, chunk_units=1 << 10, step_ms=0.5)
    a = wl.ScanSpec("chunks_a", wl.G_COSPROD, 2, np.zeros(2), np.ones(2),
                    [np.linspace(0.5, 5, 97), np.linspace(0.5, 5, 61)], 256, 3, 11)
    b = wl.ScanSpec("chunks_b", wl.G_POLY, 1, np.zeros(1), np.ones(1),
                    [np.linspace(0.5, 5, 7919)], 128, 2, 12)
    try:
        ta = srv.submit(a.integrand_id, a.N, a.lo, a.hi, a.lengths, a.values, a.samples,
                        a.trials, a.seed, 2, want_sums=True)
        tb = srv.submit(b.integrand_id, b.N, b.lo, b.hi, b.lengths, b.values, b.samples,
                        b.trials, b.seed, 0, want_sums=True)
        assert srv.wait(ta, 120000) == z.ZMC_OK and srv.wait(tb, 120000) == z.ZMC_OK
        chunks = []
        for t, spec, prec in ((ta, a, 2), (tb, b, 0)):
            res, o = srv.result(t)
            per_chunk = max(1, 1024 // (spec.trials * o.tile_splits))
            chunks.append(-(-spec.P // per_chunk))
            solo, so = z.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                              spec.values, spec.samples, spec.trials, spec.seed,
                              precision=prec, tiles=(o.tile_lanes, o.tile_splits, 256),
                              want_sums=True)
            for k in ("mean", "err", "errw", "s1", "s2"):
                assert np.array_equal(res[k], solo[k]), (spec.name, k)
        # 1024 unit-splits per chunk; a request finishes at most one chunk a step
        assert min(chunks) > 8 and srv.stats().steps >= max(chunks)
    finally:
        srv.close()


def test_large_serving_request_full_size(z):
    # The serving workload's large request at its full size (cos-product, N = 3,
    # 465 x 465 x 463 > 10^8 points, 2^12 samples x 4 trials), streamed in
    # chunks by the server: sampled points against the oracle, and every
    # output against the same scan run alone.
    spec = wl.large_scan(0)
    srv = z.Server(60 << 30)
    try:
        t = srv.submit(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                       spec.samples, spec.trials, spec.seed)
        assert srv.wait(t, 600000) == z.ZMC_OK
        res, o = srv.result(t)
        assert srv.stats().steps > 10
        pts = wl.sample_points(spec.P, 200, seed=31)
        ref = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                           spec.lengths, spec.values, spec.samples,
                                           spec.trials, spec.seed, pts, want_sums=True)
        got = {k: res[k][pts] for k in ("mean", "err", "errw")}
        V = float(np.prod(spec.hi - spec.lo))
        parity.check(got, ref, V, spec.samples, 2, spec.name + " served, sampled")
        solo = _solo(z, spec, 2, o)
        assert np.array_equal(res["mean"], solo["mean"])
        assert np.array_equal(res["err"], solo["err"])
    finally:
        srv.close()


def test_cancel_and_timeouts(z):
    srv = z.Server(1 << 30, step_ms=1.0, max_active=4)
    big = wl.scan_gauss_1e6(samples=1 << 14)  # ~0.2 s of GPU work
    try:
        t = srv.submit(big.integrand_id, big.N, big.lo, big.hi, big.lengths, big.values,
                       big.samples, big.trials, big.seed)
        assert srv.wait(t, 0) == z.ZMC_ETIMEDOUT          # bounded wait runs out
        assert z.zmc_cancel(srv.handle, t) == z.ZMC_OK
        assert srv.wait(t, 60000) == z.ZMC_ECANCELED
        assert z.zmc_cancel(srv.handle, t) == z.ZMC_EBUSY  # already finished
        s2 = srv.submit(1, 2, [0, 0], [1, 1], [4, 4], np.linspace(0.5, 5, 8), 256, 2, 9)
        assert srv.wait(s2, 60000) == z.ZMC_OK
        with pytest.raises(z.ZmcError):
            z.zmc_wait(srv.handle, 987654321, 0)
        st = srv.stats()
        assert st.cancelled == 1 and st.completed == 1
    finally:
        srv.close()


def test_injected_allocation_failures_leave_others_intact(z):
    srv = z.Server(1 << 30, fail_alloc_every=3, max_active=8)
    mix = _mix(n=12, seed=8)
    try:
        tickets = [(srv.submit(s.integrand_id, s.N, s.lo, s.hi, s.lengths, s.values, s.samples,
                               s.trials, s.seed, p), s, p) for s, p in mix]
        codes = [srv.wait(t, 60000) for t, s, p in tickets]
        assert codes.count(z.ZMC_ENOMEM) == 4 and codes.count(z.ZMC_OK) == 8, codes
        for (t, s, p), c in zip(tickets, codes):
            if c == z.ZMC_OK:
                res, o = srv.result(t)
                assert np.array_equal(res["mean"], _solo(z, s, p, o)["mean"])
    finally:
        srv.close()


def test_budget_refusal_and_shutdown_with_pending_requests(z):
    srv = z.Server(1 << 20, max_active=2)
    try:
        spec = wl.scan_gauss_1e6(samples=64)  # needs far more than 1 MiB
        with pytest.raises(z.ZmcError) as e:
            srv.submit(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                       spec.samples, spec.trials, spec.seed)
        assert e.value.status == z.ZMC_ENOMEM
        ts = [srv.submit(1, 1, [0], [1], [3], [1.0, 2.0, 3.0], 1 << 16, 2, i) for i in range(20)]
    finally:
        srv.close()  # cancels what is left; must return
