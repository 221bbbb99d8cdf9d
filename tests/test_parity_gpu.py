"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small grids run in full; the workloads at full size (the bench's launch
configuration: planner-chosen tiles, device-resident inputs) are compared on
seeded samples of grid points, which the oracle evaluates one by one.
"""
import numpy as np
import pytest

import parity
from oracle import oracle
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2]  # ZMC_FP64, ZMC_FP32, ZMC_FP32_KAHAN


@pytest.fixture(scope="module")
def zmc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc as z
    z.load()
    return z


def _oracle(spec, points=None):
    O = oracle.default()
    if points is None:
        return O.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                      spec.samples, spec.trials, spec.seed, want_sums=True)
    return O.scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                         spec.values, spec.samples, spec.trials, spec.seed, points,
                         want_sums=True)


def _gpu(z, spec, prec, **kw):
    res, out = z.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                      spec.values, spec.samples, spec.trials, spec.seed, precision=prec,
                      want_sums=True, **kw)
    return res, out


def _V(spec):
    return float(np.prod(np.asarray(spec.hi) - np.asarray(spec.lo)))


def small_cases():
    """Grids that span several blocks and end in ragged tails (S not a
    multiple of the sample group, P not a multiple of the block's units)."""
    r = np.random.default_rng(5)
    cases = []
    for N in range(1, 9):
        L = [3, 5, 2] + [1] * 5
        lens = L[:N]
        cases.append(wl.ScanSpec("cos%d" % N, wl.G_COSPROD, N, np.zeros(N), np.ones(N),
                                 [r.uniform(0.5, 5, k) for k in lens], 1003, 3, 7 + N))
        cases.append(wl.ScanSpec("gauss%d" % N, wl.G_GAUSS03, N, -np.ones(N),
                                 np.linspace(0.8, 1.2, N),
                                 [r.uniform(-1, 1, k) for k in lens], 998, 2, 100 + N))
        cases.append(wl.ScanSpec("poly%d" % N, wl.G_POLY, N, np.linspace(0, -0.5, N),
                                 np.ones(N), [r.uniform(0.5, 5, k) for k in lens], 1001, 2,
                                 2 ** 40 + N))
        cases.append(wl.ScanSpec("osc%d" % N, wl.G_OSC01, N, np.zeros(N), 2 * np.ones(N),
                                 [r.uniform(0.5, 5, k) for k in lens], 1027, 3, N))
        cases.append(wl.ScanSpec("sin%d" % N, wl.G_SINSUM, N, np.zeros(N), 3 * np.ones(N),
                                 [np.arange(7.0), np.arange(3.0)], 999, 2, 55 + N))
        cases.append(wl.ScanSpec("const%d" % N, wl.G_CONST, N, -np.ones(N), 2 * np.ones(N),
                                 [np.arange(4.0)], 1001, 2, 0))
    return cases


@pytest.mark.parametrize("prec", PRECS)
def test_small_grids_all_integrands_all_N(zmc, prec):
    for spec in small_cases():
        ref = _oracle(spec)
        got, out = _gpu(zmc, spec, prec)
        parity.check(got, ref, _V(spec), spec.samples, prec, spec.name)
        if prec == 0:
            # FP64 sums of g agree with the oracle's sequential sums closely
            sc = np.maximum(1.0, np.sqrt(ref["s2"] * spec.samples))
            assert np.all(np.abs(got["s1"] - ref["s1"]) <= 1e-12 * sc), spec.name


def test_const_integrand_exact_volume(zmc):
    spec = wl.ScanSpec("const", wl.G_CONST, 3, np.array([0.0, -2.0, 1.0]),
                       np.array([4.0, 2.0, 3.0]), [np.arange(5.0), np.arange(3.0)],
                       4096, 4, 0)
    for prec in PRECS:
        got, _ = _gpu(zmc, spec, prec)
        assert np.all(got["mean"] == 32.0), (prec, got["mean"][:4])
        assert np.all(got["err"] == 0.0)


@pytest.mark.parametrize("prec", PRECS)
def test_cosprod_100_full(zmc, prec):
    spec = wl.scan_cosprod_100()
    ref = _oracle(spec)
    got, out = _gpu(zmc, spec, prec)
    parity.check(got, ref, _V(spec), spec.samples, prec, spec.name)


@pytest.mark.parametrize("tiles", [(32, 1, 256), (8, 5, 128), (1, 3, 64), (64, 2, 256),
                                   (256, 1, 256), (512, 3, 512), (4, 1, 512)])
def test_tile_configurations_agree(zmc, tiles):
    spec = wl.scan_cosprod_100(samples=3001, trials=3)
    ref = _oracle(spec)
    for prec in PRECS:
        got, out = _gpu(zmc, spec, prec, tiles=tiles)
        assert (out.tile_lanes, out.tile_splits, out.tile_block) == tiles
        parity.check(got, ref, _V(spec), spec.samples, prec, "tiles %s" % (tiles,))


def test_same_tiles_bitwise_deterministic(zmc):
    spec = wl.scan_gauss_1e6(samples=1 << 10, trials=2)
    spec.lists = [v[:20] for v in spec.lists[:3]] + [spec.lists[3]]
    for prec in PRECS:
        a, _ = _gpu(zmc, spec, prec)
        b, _ = _gpu(zmc, spec, prec)
        assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["s2"], b["s2"])


def test_slices_reproduce_full_grid_bitwise(zmc):
    spec = wl.scan_osc_1e4(samples=1 << 10, trials=2)
    tiles = (16, 2, 256)
    full, _ = _gpu(zmc, spec, 2, tiles=tiles)
    P = spec.P
    cuts = [0, 1, 777, 4096, 9999, P]
    for a, b in zip(cuts[:-1], cuts[1:]):
        part, _ = _gpu(zmc, spec, 2, tiles=tiles, first_index=a, count=b - a)
        assert np.array_equal(part["mean"], full["mean"][a:b])
        assert np.array_equal(part["s1"], full["s1"][a:b])


def test_edge_cases(zmc):
    O = oracle.default()
    # empty slice: a valid no-op
    res, out = zmc.scan(1, 2, [0, 0], [1, 1], [3, 3], np.arange(6.0), 64, 2, 0,
                        first_index=9, count=0)
    assert res["mean"].size == 0 and out.launches == 0
    # one grid point, S = 1 (errw undefined), T = 1 (err undefined)
    res, _ = zmc.scan(5, 3, [0, 0, 0], [1, 2, 3], [1], [0.25], 1, 1, 3, precision=0)
    ref = O.scan(5, 3, [0, 0, 0], [1, 2, 3], [1], [0.25], 1, 1, 3)
    assert abs(res["mean"][0] - ref["mean"][0]) <= 1e-13 * 6
    assert np.isnan(res["err"][0]) and np.isnan(res["errw"][0])
    # sixteen parameter lists (the maximum), sine-sum of any M
    lists = [np.array([0.1 * i, 0.2 * i]) for i in range(16)]
    spec = wl.ScanSpec("m16", wl.G_SINSUM, 2, np.zeros(2), np.ones(2), lists, 257, 2, 1)
    for prec in PRECS:
        got, _ = _gpu(zmc, spec, prec, first_index=65536 - 100)
        ref = _oracle(spec, np.arange(65536 - 100, 65536))
        parity.check(got, ref, _V(spec), spec.samples, prec, "M=16")
    # a list longer than the shared-memory staging limit (global-memory path)
    spec = wl.ScanSpec("long", wl.G_SINSUM, 1, np.zeros(1), np.ones(1),
                       [np.linspace(0, 50, 6000)], 515, 2, 9)
    for prec in PRECS:
        got, _ = _gpu(zmc, spec, prec)
        parity.check(got, _oracle(spec), 1.0, spec.samples, prec, "long list")


@pytest.mark.parametrize("N", [1, 2, 4, 5, 7])
def test_every_small_sample_count(zmc, N):
    # S = 1 .. 12 covers samples fewer than one group, exactly one group, a
    # group plus a ragged tail and (N = 5) single-sample groups; the sums must
    # match the oracle's, and the tile shape (one lane or 32 lanes, one or
    # several sample ranges) must not matter beyond summation order.
    lists = [np.linspace(0.5, 5.0, 3 + k) for k in range(min(N, 3))] + [[1.0]] * max(0, N - 3)
    for S in range(1, 13):
        spec = wl.ScanSpec("S%d" % S, wl.G_COSPROD, N, np.zeros(N), np.ones(N), lists, S, 3, S)
        ref = _oracle(spec)
        for prec in PRECS:
            for tiles in [(0, 0, 0), (1, 1, 64), (32, 2, 128)]:
                got, _ = _gpu(zmc, spec, prec, tiles=tiles)
                V = _V(spec)
                scale = V * np.maximum(1.0, np.sqrt(np.mean(ref["s2"], axis=1) / S))
                tol = (1e-12 if prec == 0 else 1e-5) * scale
                assert np.all(np.abs(got["mean"] - ref["mean"]) <= tol), (N, S, prec, tiles)
                assert np.allclose(got["s1"], ref["s1"], rtol=0, atol=(1e-12 if prec == 0 else 1e-5) * S)


@pytest.mark.parametrize("prec", [0, 2])
def test_maximum_samples_per_point(zmc, prec):
    # The largest S the budget allows at N = 8 (S*N = 2^34 - 2^20): Philox call
    # indices reach 3.4e9 and the last group holds one sample.  The estimate
    # agrees with the closed form within its standard error, the pooled error
    # matches the closed-form one, and the last call's words equal the
    # oracle's.
    import closed_forms as cf
    N, S = 8, 2 ** 31 - 2 ** 17
    x = 0.3
    lo, hi = np.zeros(N), np.ones(N)
    res, out = zmc.scan(5, N, lo, hi, [1], [x], S, 2, 11, precision=prec, want_sums=True)
    f = cf.integral(cf.G_SINSUM, [x], lo, hi)
    se = cf.sigma_I(cf.G_SINSUM, [x], lo, hi, S) / np.sqrt(2)
    assert abs(res["mean"][0] - f) < 5 * se, (res["mean"][0], f, se)
    assert 0.9 < res["errw"][0] / se < 1.1
    last_call = (S * N - 1) // 5
    words = zmc.zmc_stream_words(11, 0, 1, 4 * last_call, 4)
    O = oracle.default()
    assert list(words) == [O.word(11, 0, 1, 4 * last_call + i) for i in range(4)]


def test_grid_index_beyond_32_bits(zmc):
    big = 70000  # P = 4.9e9 > 2^32: the high counter word of p is non-zero
    spec = wl.ScanSpec("big", wl.G_GAUSS03, 2, -np.ones(2), np.ones(2),
                       [np.linspace(-1, 1, big), np.linspace(-1, 1, big)], 509, 3,
                       2 ** 63 + 5)
    first = 2 ** 32 - 40
    for prec in PRECS:
        got, _ = _gpu(zmc, spec, prec, first_index=first, count=100)
        ref = _oracle(spec, np.arange(first, first + 100))
        parity.check(got, ref, 4.0, spec.samples, prec, "p > 2^32")


def test_stream_words_match_oracle(zmc):
    O = oracle.default()
    for seed, p, t, w0, n in [(0, 0, 0, 0, 64), (2 ** 64 - 1, 2 ** 40 + 3, 7, 2 ** 33, 99),
                              (12345, 999, 2 ** 31 - 1, 5, 257)]:
        got = zmc.zmc_stream_words(seed, p, t, w0, n)
        want = np.array([O.word(seed, p, t, w0 + i) for i in range(n)], dtype=np.uint32)
        assert np.array_equal(got, want)


def test_device_memory_path_matches_host_path(zmc):
    import torch
    spec = wl.scan_gauss_1e6(samples=512, trials=2)
    spec.lists = [v[:30] for v in spec.lists[:3]] + [spec.lists[3]]
    host, _ = _gpu(zmc, spec, 2)
    vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
    P = spec.P
    mean = torch.empty(P, dtype=torch.float64, device="cuda")
    err = torch.empty_like(mean)
    s = torch.cuda.current_stream()
    zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                    spec.samples, spec.trials, spec.seed, mean, err,
                    stream=s.cuda_stream)
    s.synchronize()
    assert np.array_equal(mean.cpu().numpy(), host["mean"])
    # caller-provided workspace: the library allocates nothing
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, mem=zmc.ZMC_MEM_DEVICE)
    nbytes = zmc.zmc_workspace_size(d)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    mean2 = torch.empty_like(mean)
    zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                    spec.samples, spec.trials, spec.seed, mean2, err, workspace=ws,
                    stream=s.cuda_stream)
    s.synchronize()
    assert torch.equal(mean, mean2)
    # host pointers in device mode are refused
    with pytest.raises(zmc.ZmcError):
        zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                        spec.samples, spec.trials, spec.seed, np.empty(P), err)


# ------------------------------------------- full-size workloads, sampled --
def _full_device(zmc, spec, prec):
    import torch
    vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
    mean = torch.empty(spec.P, dtype=torch.float64, device="cuda")
    err = torch.empty_like(mean)
    errw = torch.empty_like(mean)
    s = torch.cuda.current_stream()
    zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                    spec.samples, spec.trials, spec.seed, mean, err, errw,
                    precision=prec, stream=s.cuda_stream)
    s.synchronize()
    return {"mean": mean.cpu().numpy(), "err": err.cpu().numpy(),
            "errw": errw.cpu().numpy()}


@pytest.mark.parametrize("prec", [2, 1, 0])
def test_gauss_1e6_full_size_sampled(zmc, prec):
    spec = wl.scan_gauss_1e6()
    got = _full_device(zmc, spec, prec)
    pts = wl.sample_points(spec.P, 48 if prec else 16)
    ref = _oracle(spec, pts)
    sub = {k: v[pts] for k, v in got.items()}
    parity.check(sub, ref, _V(spec), spec.samples, prec, spec.name)
    assert np.all(np.isfinite(got["mean"])) and np.all(got["err"] > 0)


@pytest.mark.parametrize("prec", [2, 1, 0])
def test_osc_1e4_full_size_sampled(zmc, prec):
    """The precision-stress workload at full size (10^4 points x 8 trials x
    2^20 samples) in FP32-Kahan, plain FP32 and FP64, on sampled points."""
    spec = wl.scan_osc_1e4()
    got = _full_device(zmc, spec, prec)
    pts = wl.sample_points(spec.P, 24 if prec else 16)
    ref = _oracle(spec, pts)
    sub = {k: v[pts] for k, v in got.items()}
    parity.check(sub, ref, _V(spec), spec.samples, prec, spec.name)


@pytest.mark.parametrize("prec", [2, 1, 0])
def test_registry_scans_at_scale_sampled(zmc, prec):
    """Every (integrand, N) of the registry at the sweep's scale (FP32-Kahan and
    FP32: 10^5 points x 4 trials x 2^15 samples; FP64: 2 x 10^4 points) with
    the planner's tiles, against the oracle on 4 seeded points per scan."""
    for gid in (1, 2, 3, 4, 5):
        for N in range(1, 9):
            spec = wl.registry_scan(gid, N, points=10 ** 5 if prec else 2 * 10 ** 4)
            got = _full_device(zmc, spec, prec)
            pts = wl.sample_points(spec.P, 4, seed=100 * gid + N)
            ref = _oracle(spec, pts)
            sub = {k: v[pts] for k, v in got.items()}
            parity.check(sub, ref, _V(spec), spec.samples, prec, spec.name)
