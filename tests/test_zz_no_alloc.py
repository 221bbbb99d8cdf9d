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


def _run(zmc, torch, spec, noalloc):
    vals, out = _buffers(torch, spec)
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, zmc.ZMC_FP32_KAHAN,
                            mem=zmc.ZMC_MEM_DEVICE, flags=zmc.ZMC_F_SYNC)
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
