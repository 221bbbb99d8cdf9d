"""The checking build (libzmc_debug.so, ZMC_DEBUG=1) on small cases.

Every kernel of that build checks its grid indices, list digits and offsets,
staged-table slots, batch tiles and partial-sum slots before the access and
records a failure on the device instead of trapping.  Here it runs every
integrand at N = 1..8 in every precision on small grids (P <= 16 points,
S <= 64 samples), a batch and a served request, with parity against the
oracle, and no check may fail.  Nothing is injected on the device.

The library runs in a child pytest process (ZMC_LIBRARY names the debug
build), so this process's release library is untouched.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import parity
from oracle import oracle
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
IN_CHILD = os.environ.get("ZMC_DEBUG_CHILD") == "1"


def _small_cases():
    r = np.random.default_rng(17)
    cases = []
    for N in range(1, 9):
        lens = ([3, 2, 2] + [1] * 5)[:N]     # P <= 12
        for gid in range(6):
            if gid == wl.G_GAUSS03:
                lists, lo, hi = [r.uniform(-1, 1, k) for k in lens], -np.ones(N), np.ones(N)
            elif gid in (wl.G_CONST, wl.G_SINSUM):
                lists, lo, hi = [np.arange(4.0), np.arange(3.0)], np.zeros(N), 2 * np.ones(N)
            else:
                lists, lo, hi = [r.uniform(0.5, 5, k) for k in lens], np.zeros(N), np.ones(N)
            S = int(r.integers(1, 65))
            cases.append(wl.ScanSpec("dbg_g%d_N%d" % (gid, N), gid, N, lo, hi, lists, S,
                                     int(r.integers(1, 4)), 300 + 10 * N + gid))
    return cases


@pytest.mark.skipif(not IN_CHILD, reason="runs inside the debug-build child process")
def test_in_debug_process_every_kernel_passes_its_checks():
    import torch
    from paper_1910_01965_gb300 import zmc
    assert torch.cuda.is_available()
    zmc.load()
    assert zmc.LIBRARY.endswith("libzmc_debug.so")
    assert zmc.zmc_debug_failures()[0] == 0            # a checking build, nothing failed yet
    O = oracle.default()
    for spec in _small_cases():
        assert spec.P <= 16 and spec.samples <= 64
        ref = O.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                     spec.samples, spec.trials, spec.seed, want_sums=True)
        V = float(np.prod(spec.hi - spec.lo))
        for prec in (0, 1, 2):
            for tiles in [(0, 0, 0), (4, 3, 64)]:
                got, out = zmc.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                    spec.values, spec.samples, spec.trials, spec.seed,
                                    precision=prec, tiles=tiles, chunk_points=5)
                parity.check(got, ref, V, spec.samples, prec, spec.name)
    # one batch of mixed scans and one served request
    specs = _small_cases()[::7]
    descs, outs, keep = [], [], []
    for i, spec in enumerate(specs):
        d, k = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                             spec.values, spec.samples, spec.trials, spec.seed, i % 3)
        res = {"mean": np.empty(spec.P), "err": np.empty(spec.P)}
        o = zmc.zmc_scan_out()
        o.mean, o.err = zmc._ptr(res["mean"]), zmc._ptr(res["err"])
        descs.append(d)
        outs.append(o)
        keep.append((k, res))
    zmc.zmc_scan_batch(descs, outs)
    srv = zmc.Server(1 << 30)
    try:
        spec = specs[0]
        t = srv.submit(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                       spec.samples, spec.trials, spec.seed)
        srv.wait(t)
    finally:
        srv.close()
    n, code, index = zmc.zmc_debug_failures()
    assert n == 0, (n, code, index)


def test_debug_build_runs_clean_on_small_cases():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import build
    lib = build.build_debug()
    env = dict(os.environ, ZMC_LIBRARY=lib, ZMC_DEBUG_CHILD="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.abspath(__file__), "-q", "-x",
                        "-p", "no:cacheprovider", "-k", "in_debug_process"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert "1 passed" in r.stdout, r.stdout[-2000:]
