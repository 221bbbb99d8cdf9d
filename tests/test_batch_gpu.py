"""Many scans in one persistent launch (zmc_batch.h) through the C ABI.

Each scan of a batch must equal the same scan run alone with the same tile
configuration bit for bit (same stream, same per-unit sums, same fixed-order
reductions), and must match the FP64 oracle within the parity tolerances.
"""
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


def _V(spec):
    return float(np.prod(np.asarray(spec.hi) - np.asarray(spec.lo)))


def mixed_specs():
    r = np.random.default_rng(9)
    specs, precs = [], []
    for i, (gid, N) in enumerate([(1, 1), (2, 4), (3, 3), (4, 6), (5, 2), (0, 2), (1, 8),
                                  (2, 7), (3, 5), (4, 2), (2, 1), (1, 3)]):
        lens = [int(r.integers(1, 7)) for _ in range(N)] if gid in (1, 2, 3, 4) else [5, 3]
        if gid == 2:
            lists, lo, hi = [r.uniform(-1, 1, L) for L in lens], -np.ones(N), np.ones(N)
        else:
            lists, lo, hi = [r.uniform(0.5, 5, L) for L in lens], np.zeros(N), np.linspace(1, 2, N)
        S = int(r.integers(200, 3000))
        specs.append(wl.ScanSpec("mix%d" % i, gid, N, lo, hi, lists, S, int(r.integers(2, 5)),
                                 1000 + i))
        precs.append([2, 1, 0][i % 3])
    return specs, precs


def _host_descs(z, specs, precs):
    keep, descs, outs, res = [], [], [], []
    for spec, prec in zip(specs, precs):
        d, k = z.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                           spec.values, spec.samples, spec.trials, spec.seed, prec)
        keep.append(k)
        r = {"mean": np.empty(spec.P), "err": np.empty(spec.P), "errw": np.empty(spec.P),
             "s1": np.empty((spec.P, spec.trials)), "s2": np.empty((spec.P, spec.trials))}
        o = z.zmc_scan_out()
        o.mean, o.err, o.errw = z._ptr(r["mean"]), z._ptr(r["err"]), z._ptr(r["errw"])
        o.s1, o.s2 = z._ptr(r["s1"]), z._ptr(r["s2"])
        descs.append(d)
        outs.append(o)
        res.append(r)
    return descs, outs, res, keep


def test_mixed_batch_matches_oracle_and_solo_runs(z):
    specs, precs = mixed_specs()
    descs, outs, res, keep = _host_descs(z, specs, precs)
    outs = z.zmc_scan_batch(descs, outs)
    O = oracle.default()
    for spec, prec, r, o in zip(specs, precs, res, outs):
        ref = O.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                     spec.samples, spec.trials, spec.seed, want_sums=True)
        parity.check(r, ref, _V(spec), spec.samples, prec, spec.name + " in batch")
        solo, so = z.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                          spec.values, spec.samples, spec.trials, spec.seed, precision=prec,
                          tiles=(o.tile_lanes, o.tile_splits, 256), want_sums=True)
        assert np.array_equal(solo["s1"], r["s1"]) and np.array_equal(solo["mean"], r["mean"]), \
            spec.name


def test_batch_object_graph_replays_are_identical(z):
    import torch
    specs, precs = mixed_specs()
    descs, outs, bufs, keep = [], [], [], []
    for spec, prec in zip(specs, precs):
        vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
        d, k = z.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                           spec.samples, spec.trials, spec.seed, prec, mem=z.ZMC_MEM_DEVICE)
        m = torch.empty(spec.P, dtype=torch.float64, device="cuda")
        e = torch.empty_like(m)
        o = z.zmc_scan_out()
        o.mean, o.err = z._ptr(m), z._ptr(e)
        descs.append(d)
        outs.append(o)
        bufs.append((m, e))
        keep.append((k, vals))
    h = z.zmc_batch_create(descs, outs, z.ZMC_BATCH_GRAPH)
    try:
        info = z.zmc_batch_info_get(h)
        assert info.graph == 1 and info.scans == len(specs) and info.precisions == 3
        s = torch.cuda.current_stream()
        z.zmc_batch_run(h, s.cuda_stream)
        s.synchronize()
        first = [m.clone() for m, e in bufs]
        for m, e in bufs:
            m.zero_()
        z.zmc_batch_run(h, s.cuda_stream)
        s.synchronize()
        for a, (m, e) in zip(first, bufs):
            assert torch.equal(a, m)
    finally:
        z.zmc_batch_destroy(h)
    # the one-shot host batch gives the same numbers
    hd, ho, hres, hkeep = _host_descs(z, specs, precs)
    z.zmc_scan_batch(hd, ho)
    for a, r in zip(first, hres):
        assert np.array_equal(a.cpu().numpy(), r["mean"])


def test_batch_with_empty_slices_and_validation(z):
    specs, precs = mixed_specs()
    specs, precs = specs[:3], precs[:3]
    descs, outs, res, keep = _host_descs(z, specs, precs)
    descs[1].first_index = specs[1].P
    descs[1].count = 0
    z.zmc_scan_batch(descs, outs)
    O = oracle.default()
    for i in (0, 2):
        spec = specs[i]
        ref = O.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                     spec.samples, spec.trials, spec.seed, want_sums=True)
        parity.check(res[i], ref, _V(spec), spec.samples, precs[i], spec.name)
    bad, bo, _, k2 = _host_descs(z, specs[:2], precs[:2])
    bad[1].mem = z.ZMC_MEM_DEVICE
    with pytest.raises(z.ZmcError):
        z.zmc_scan_batch(bad, bo)


def test_uneven_256_batch_sampled_against_oracle(z):
    import torch
    specs = wl.batch_uneven_256()
    descs, outs, bufs, keep = [], [], [], []
    for spec in specs:
        vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
        d, k = z.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                           spec.samples, spec.trials, spec.seed, z.ZMC_FP32_KAHAN,
                           mem=z.ZMC_MEM_DEVICE)
        m = torch.empty(spec.P, dtype=torch.float64, device="cuda")
        e = torch.empty_like(m)
        w = torch.empty_like(m)
        o = z.zmc_scan_out()
        o.mean, o.err, o.errw = z._ptr(m), z._ptr(e), z._ptr(w)
        descs.append(d)
        outs.append(o)
        bufs.append((m, e, w))
        keep.append((k, vals))
    h = z.zmc_batch_create(descs, outs, z.ZMC_BATCH_GRAPH)
    try:
        z.zmc_batch_run(h, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    finally:
        z.zmc_batch_destroy(h)
    O = oracle.default()
    rng = np.random.default_rng(3)
    for i in rng.choice(len(specs), 24, replace=False):
        spec = specs[i]
        pts = wl.sample_points(spec.P, 4, seed=int(i))
        ref = O.scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                            spec.values, spec.samples, spec.trials, spec.seed, pts,
                            want_sums=True)
        m, e, w = bufs[i]
        got = {"mean": m.cpu().numpy()[pts], "err": e.cpu().numpy()[pts],
               "errw": w.cpu().numpy()[pts]}
        parity.check(got, ref, _V(spec), spec.samples, z.ZMC_FP32_KAHAN, spec.name)
