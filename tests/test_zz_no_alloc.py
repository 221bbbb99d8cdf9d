"""zmc_scan_noalloc against zmc_scan_ex, through the C ABI.

zmc_scan_noalloc exists for callers that cannot allocate device memory when
they scan (latency-critical loops where an allocation can wait on the driver,
hosts whose device memory is owned and budgeted by another allocator, hosts
with a footprint fixed at start-up).  It must give the same results as the
allocating entry point, call after call, since every call reuses one fixed
scratch array.  This file is named to run after the other tests.
"""
import numpy as np
import pytest

import parity
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc
    zmc.load()
    return zmc, torch


def _buffers(torch, spec):
    dev = "cuda"
    vals = torch.tensor(spec.values, dtype=torch.float64, device=dev)
    n = spec.P
    out = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in ("mean", "err", "errw")}
    out["s1"] = torch.empty((n, spec.trials), dtype=torch.float64, device=dev)
    out["s2"] = torch.empty((n, spec.trials), dtype=torch.float64, device=dev)
    return vals, out


def _out_struct(zmc, out):
    o = zmc.zmc_scan_out()
    o.mean, o.err, o.errw = zmc._ptr(out["mean"]), zmc._ptr(out["err"]), zmc._ptr(out["errw"])
    o.s1, o.s2 = zmc._ptr(out["s1"]), zmc._ptr(out["s2"])
    return o


def _run(zmc, torch, spec, noalloc, tiles=(0, 0, 0)):
    vals, out = _buffers(torch, spec)
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, zmc.ZMC_FP32_KAHAN,
                            mem=zmc.ZMC_MEM_DEVICE, flags=zmc.ZMC_F_SYNC, tiles=tiles)
    o = _out_struct(zmc, out)
    if noalloc:
        zmc.zmc_scan_noalloc(d, o)
    else:
        zmc.zmc_scan_ex(d, o)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, o


def _specs():
    gauss = wl.scan_gauss_1e6(samples=1 << 12)
    gauss.lists[0] = gauss.lists[0][:10]          # 10 x 100 x 100 x 1 grid
    osc = wl.scan_osc_1e4(samples=1 << 13, trials=3)
    return [gauss, osc]


def test_noalloc_matches_scan_ex_on_two_calls_in_a_row(env):
    zmc, torch = env
    for spec in _specs():                          # two calls, different shapes
        ref, _ = _run(zmc, torch, spec, noalloc=False)
        got, o = _run(zmc, torch, spec, noalloc=True)
        assert o.launches == 2
        V = float(np.prod(np.asarray(spec.hi) - np.asarray(spec.lo)))
        parity.check(got, ref, V, spec.samples, zmc.ZMC_FP32_KAHAN, spec.name + " noalloc")


def test_noalloc_equals_scan_ex_bitwise_with_the_same_plan(env):
    """Both entry points plan the same tiles (given or left open), so their
    results agree bit for bit."""
    zmc, torch = env
    spec = _specs()[1]
    for tiles in [(0, 0, 0), (16, 3, 128)]:
        ref, o1 = _run(zmc, torch, spec, noalloc=False, tiles=tiles)
        got, o2 = _run(zmc, torch, spec, noalloc=True, tiles=tiles)
        assert (o1.tile_lanes, o1.tile_splits, o1.tile_block) == \
            (o2.tile_lanes, o2.tile_splits, o2.tile_block)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (tiles, k)


def _device_memory(torch):
    """(free device bytes, the default pool's reserved and used bytes)."""
    import ctypes
    rt = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    vals = []
    for attr in (5, 7):   # cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent
        v = ctypes.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        vals.append(v.value)
    free, _ = torch.cuda.mem_get_info()
    return (free, *vals)


def test_noalloc_allocates_no_device_memory(env):
    """After a warm-up call of each shape (which loads the module holding the
    scratch array and the kernels), calls of two different shapes leave the
    device's free memory and the stream-ordered pool unchanged."""
    zmc, torch = env
    specs = _specs()
    prepared = []
    for spec in specs:
        vals, out = _buffers(torch, spec)
        d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                vals, spec.samples, spec.trials, spec.seed, zmc.ZMC_FP32_KAHAN,
                                mem=zmc.ZMC_MEM_DEVICE, flags=zmc.ZMC_F_SYNC)
        prepared.append((d, keep, vals, out, _out_struct(zmc, out)))
    for d, keep, vals, out, o in prepared:   # warm-up: loads each shape's kernels
        zmc.zmc_scan_noalloc(d, o)
    torch.cuda.synchronize()
    before = _device_memory(torch)
    for d, keep, vals, out, o in prepared + prepared:
        zmc.zmc_scan_noalloc(d, o)
    torch.cuda.synchronize()
    assert _device_memory(torch) == before


def test_noalloc_at_its_scratch_boundary(env):
    """Partial sums of exactly 16 MiB (2^18 points x 4 trials x 1 split x
    16 bytes) fit; one more point does not."""
    zmc, torch = env
    spec = wl.scan_gauss_1e6(samples=40)
    spec.lists = [np.linspace(-1, 1, 512), np.linspace(-1, 1, 512), np.zeros(1), np.zeros(1)]
    assert spec.P * spec.trials * 16 == zmc.ZMC_NOALLOC_SCRATCH_BYTES
    ref, _ = _run(zmc, torch, spec, noalloc=False, tiles=(8, 1, 256))
    got, o = _run(zmc, torch, spec, noalloc=True, tiles=(8, 1, 256))
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    spec.lists[2] = np.zeros(2)      # 2^19 points: twice the scratch
    vals, out = _buffers(torch, spec)
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, zmc.ZMC_FP32_KAHAN,
                            mem=zmc.ZMC_MEM_DEVICE, tiles=(8, 1, 256),
                            first_index=0, count=(1 << 18) + 1)
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_scan_noalloc(d, _out_struct(zmc, out))
    assert e.value.status == zmc.ZMC_EINVAL and "scratch" in str(e.value)


def test_noalloc_plan_only_computes_nothing(env):
    zmc, torch = env
    spec = _specs()[1]
    vals, out = _buffers(torch, spec)
    out["mean"].fill_(7.0)
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, zmc.ZMC_FP32_KAHAN,
                            mem=zmc.ZMC_MEM_DEVICE, flags=zmc.ZMC_F_PLAN_ONLY)
    o = _out_struct(zmc, out)
    zmc.zmc_scan_noalloc(d, o)
    torch.cuda.synchronize()
    assert o.launches == 0 and o.tile_lanes > 0
    assert bool((out["mean"] == 7.0).all())


def test_noalloc_rejects_requests_beyond_its_scratch(env):
    zmc, torch = env
    spec = wl.scan_gauss_1e6(samples=64)           # 1e6 points x 4 trials x 16 B > 16 MiB
    vals, out = _buffers(torch, spec)
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, zmc.ZMC_FP32_KAHAN,
                            mem=zmc.ZMC_MEM_DEVICE)
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_scan_noalloc(d, _out_struct(zmc, out))
    assert e.value.status == zmc.ZMC_EINVAL and "scratch" in str(e.value)
