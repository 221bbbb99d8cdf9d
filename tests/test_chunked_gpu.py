"""zmc_scan_ex cut into chunks of consecutive grid points (Sec. 2's batches).

Every chunk runs the tile plan of the whole call, so a scan cut into many
chunks equals the one-chunk scan bit for bit, in device memory and in host
memory (pinned arrays written by the copy stream directly, pageable ones
through the library's staging buffers).  Grids beyond 2^32 points and calls
that need more than 2^31 - 1 blocks in total run through the same call.
"""
import numpy as np
import pytest

import parity
from oracle import oracle
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zmc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc as z
    z.load()
    return z


def _spec():
    r = np.random.default_rng(21)
    return wl.ScanSpec("gauss_chunks", wl.G_GAUSS03, 4, -np.ones(4), np.ones(4),
                       [r.uniform(-1, 1, 37), r.uniform(-1, 1, 29), r.uniform(-1, 1, 11),
                        np.zeros(1)], 999, 3, 5)


def _host(z, spec, prec, chunk_points, pinned=False, first=0, count=-1, tiles=(0, 0, 0)):
    import torch
    n = (spec.P - first) if count < 0 else count
    T = spec.trials

    def buf(shape):
        if pinned:
            return torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
        return np.empty(shape)
    res = {"mean": buf(n), "err": buf(n), "errw": buf(n), "s1": buf((n, T)), "s2": buf((n, T))}
    d, keep = z.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                          spec.values, spec.samples, spec.trials, spec.seed, prec,
                          first_index=first, count=count, tiles=tiles,
                          chunk_points=chunk_points)
    o = z.zmc_scan_out()
    for k in res:
        setattr(o, k, z._ptr(res[k]))
    z.zmc_scan_ex(d, o)
    return res, o


@pytest.mark.parametrize("prec", [2, 0])
def test_forced_chunks_equal_one_chunk_bitwise_host(zmc, prec):
    spec = _spec()                       # 11,803 points
    one, o1 = _host(zmc, spec, prec, chunk_points=0)
    assert o1.chunks == 1
    for cp, pinned in [(3001, False), (3001, True), (977, False), (1, False)]:
        if cp == 1:   # a slice, one point per chunk, with the whole grid's tiles
            got, o = _host(zmc, spec, prec, chunk_points=1, first=5000, count=9,
                           tiles=(o1.tile_lanes, o1.tile_splits, o1.tile_block))
            ref = {k: v[5000:5009] for k, v in one.items()}
            assert o.chunks == 9
        else:
            got, o = _host(zmc, spec, prec, chunk_points=cp, pinned=pinned)
            ref = one
            assert o.chunks == -(-spec.P // cp) and o.chunks >= 4
        assert (o.tile_lanes, o.tile_splits, o.tile_block) == \
            (o1.tile_lanes, o1.tile_splits, o1.tile_block)
        assert o.launches == 2 * o.chunks
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (cp, pinned, k)


def test_forced_chunks_equal_one_chunk_bitwise_device(zmc):
    import torch
    spec = _spec()
    vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
    outs = []
    for cp in (0, 4000, 1234):
        m = torch.empty(spec.P, dtype=torch.float64, device="cuda")
        e, w = torch.empty_like(m), torch.empty_like(m)
        s1 = torch.empty((spec.P, spec.trials), dtype=torch.float64, device="cuda")
        s2 = torch.empty_like(s1)
        o = zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, m, e, w, s1, s2,
                            flags=zmc.ZMC_F_SYNC | zmc.ZMC_F_TIMINGS, chunk_points=cp)
        assert o.chunks == (1 if cp == 0 else -(-spec.P // cp))
        assert o.kernel_ms > 0 and o.d2h_ms == 0
        outs.append([t.cpu() for t in (m, e, w, s1, s2)])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert torch.equal(a, b)
    # a caller workspace sized by zmc_workspace_size for the chunked call
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, mem=zmc.ZMC_MEM_DEVICE,
                            chunk_points=1234)
    nb = zmc.zmc_workspace_size(d)
    d0, keep0 = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                              spec.samples, spec.trials, spec.seed, mem=zmc.ZMC_MEM_DEVICE)
    assert nb < zmc.zmc_workspace_size(d0)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    m = torch.empty(spec.P, dtype=torch.float64, device="cuda")
    e = torch.empty_like(m)
    zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                    spec.samples, spec.trials, spec.seed, m, e, workspace=ws,
                    flags=zmc.ZMC_F_SYNC, chunk_points=1234)
    assert torch.equal(m.cpu(), outs[0][0])


def test_default_chunking_of_a_large_host_scan_overlaps_copies(zmc):
    """2^23 points in host memory: the library cuts the slice into 8 chunks
    and the copies of results run beside later chunks' sampling."""
    spec = wl.ScanSpec("cos_2^23", wl.G_COSPROD, 3, np.zeros(3), np.ones(3),
                       [np.linspace(0.5, 5, 256), np.linspace(0.5, 5, 256),
                        np.linspace(0.5, 5, 128)], 200, 2, 3)
    assert spec.P == 1 << 23
    got, o = _host(zmc, spec, 2, chunk_points=0)
    assert o.chunks == 8
    one, o1 = _host(zmc, spec, 2, chunk_points=spec.P)
    assert o1.chunks == 1
    for k in got:
        assert np.array_equal(got[k], one[k]), k
    pts = wl.sample_points(spec.P, 24, seed=9)
    ref = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                       spec.lengths, spec.values, spec.samples, spec.trials,
                                       spec.seed, pts, want_sums=True)
    parity.check({k: got[k][pts] for k in ("mean", "err", "errw")}, ref, 1.0, spec.samples,
                 2, spec.name)


@pytest.mark.parametrize("prec", [2, 0])
def test_grid_beyond_2_32_points_chunked_sampled_against_oracle(zmc, prec):
    """P = 2048 x 2048 x 1025 > 2^32; a slice of 2^22 points across 2^32, cut
    into 16 chunks, against the oracle on sampled points."""
    r = np.random.default_rng(8)
    spec = wl.ScanSpec("cos_P_gt_2^32", wl.G_COSPROD, 3, np.zeros(3), np.ones(3),
                       [r.uniform(0.5, 5, 2048), r.uniform(0.5, 5, 2048),
                        r.uniform(0.5, 5, 1025)], 96, 2, 77)
    assert spec.P > 1 << 32
    first, count = (1 << 32) - (1 << 21), 1 << 22
    got, o = _host(zmc, spec, prec, chunk_points=1 << 18, first=first, count=count)
    assert o.chunks == 16
    loc = wl.sample_points(count, 40, seed=3)
    loc = np.unique(np.concatenate([loc, [(1 << 21) - 1, 1 << 21]]))  # both sides of 2^32
    ref = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                       spec.lengths, spec.values, spec.samples, spec.trials,
                                       spec.seed, first + loc, want_sums=True)
    parity.check({k: got[k][loc] for k in ("mean", "err", "errw")}, ref, 1.0, spec.samples,
                 prec, spec.name)
    for k in ("s1", "s2"):
        assert np.allclose(got[k][loc], ref[k], rtol=1e-12 if prec == 0 else 1e-5,
                           atol=1e-12 if prec == 0 else 1e-4)


def test_more_than_2_31_blocks_in_one_call(zmc):
    """One unit-split per 64-thread block and 2^22 + 1 points x 512 trials:
    2^31 + 512 blocks in total, which no single launch takes; the call cuts
    them into chunks and matches the oracle on sampled points."""
    import torch
    spec = wl.ScanSpec("poly_many_blocks", wl.G_POLY, 1, np.zeros(1), np.ones(1),
                       [np.linspace(0.5, 5, (1 << 22) + 1)], 5, 512, 11)
    vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
    m = torch.empty(spec.P, dtype=torch.float64, device="cuda")
    e, w = torch.empty_like(m), torch.empty_like(m)
    o = zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                        spec.samples, spec.trials, spec.seed, m, e, w, tiles=(64, 1, 64),
                        flags=zmc.ZMC_F_SYNC)
    assert spec.P * spec.trials > (1 << 31) - 1 and o.chunks > 1
    pts = wl.sample_points(spec.P, 64, seed=4)
    ref = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                       spec.lengths, spec.values, spec.samples, spec.trials,
                                       spec.seed, pts, want_sums=True)
    got = {"mean": m.cpu().numpy()[pts], "err": e.cpu().numpy()[pts],
           "errw": w.cpu().numpy()[pts]}
    parity.check(got, ref, 1.0, spec.samples, 2, spec.name)


@pytest.mark.parametrize("pinned", [False, True])
def test_chunked_host_scan_with_only_mean_and_err_and_timings(zmc, pinned):
    """The optional outputs left NULL, timings on, chunk_points beyond the
    slice (one chunk) and a ragged last chunk: the same bits as one chunk,
    and the exposed copy time is what is left after the last chunk."""
    import torch
    spec = _spec()

    def run(cp):
        if pinned:
            m = torch.empty(spec.P, dtype=torch.float64).pin_memory().numpy()
            e = torch.empty(spec.P, dtype=torch.float64).pin_memory().numpy()
        else:
            m, e = np.empty(spec.P), np.empty(spec.P)
        d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                spec.values, spec.samples, spec.trials, spec.seed, 2,
                                flags=zmc.ZMC_F_TIMINGS, chunk_points=cp)
        o = zmc.zmc_scan_out()
        o.mean, o.err = zmc._ptr(m), zmc._ptr(e)
        zmc.zmc_scan_ex(d, o)
        return m, e, o
    m1, e1, o1 = run(10 * spec.P)
    assert o1.chunks == 1
    m5, e5, o5 = run(2500)                  # 5 chunks, the last one ragged
    assert o5.chunks == 5 and o5.launches == 10
    assert np.array_equal(m1, m5) and np.array_equal(e1, e5)
    assert o5.kernel_ms > 0 and o5.finalize_ms > 0 and 0 <= o5.d2h_ms <= o5.total_ms


def test_chunk_counts_of_empty_and_plan_only_calls(zmc):
    """An empty slice runs no chunk; ZMC_F_PLAN_ONLY reports the chunks a call
    would take without computing."""
    spec = _spec()
    res, o = zmc.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                      spec.samples, spec.trials, spec.seed, first_index=spec.P, count=0,
                      chunk_points=5)
    assert o.chunks == 0 and o.launches == 0
    res, o = zmc.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                      spec.samples, spec.trials, spec.seed, chunk_points=1000,
                      flags=zmc.ZMC_F_PLAN_ONLY)
    assert o.chunks == -(-spec.P // 1000) and o.launches == 0
