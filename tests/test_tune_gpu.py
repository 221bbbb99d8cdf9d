"""The tile autotuner (zmc_tune.h): a timed search over lanes, block and
per-lane work whose winner the planners then use."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import parity
from oracle import oracle
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def z():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc
    zmc.load()
    zmc.zmc_autotune_reset()
    yield zmc
    zmc.zmc_autotune_reset()


def test_tuned_plan_is_used_and_stays_in_tolerance(z):
    spec = wl.scan_osc_1e4(samples=1 << 14, trials=4)
    d, keep = z.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                          spec.values, spec.samples, spec.trials, spec.seed)
    r = z.zmc_autotune(d, 400)
    assert r.candidates >= 2 and r.lanes & (r.lanes - 1) == 0 and r.block in (128, 256, 512)
    assert r.evals_per_s >= 0.99 * r.default_evals_per_s > 0
    got = z.zmc_autotune_lookup(z.ZMC_FP32_KAHAN, spec.integrand_id, spec.N, spec.samples)
    assert got is not None and (got.lanes, got.block) == (r.lanes, r.block)
    res, o = z.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                    spec.samples, spec.trials, spec.seed, want_sums=True)
    assert (o.tile_lanes, o.tile_block) == (r.lanes, r.block)
    pts = wl.sample_points(spec.P, 16)
    ref = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                       spec.lengths, spec.values, spec.samples, spec.trials,
                                       spec.seed, pts, want_sums=True)
    sub = {k: v[pts] for k, v in res.items() if k in ("mean", "err", "errw")}
    parity.check(sub, ref, float(np.prod(spec.hi - spec.lo)), spec.samples, 2, "tuned")
    z.zmc_autotune_reset()
    assert z.zmc_autotune_lookup(z.ZMC_FP32_KAHAN, spec.integrand_id, spec.N,
                                 spec.samples) is None


CHILD = r"""
import json, sys
sys.path.insert(0, %r)
from paper_1910_01965_gb300 import zmc
zmc.load()
mode = sys.argv[1]
if mode == "tune":
    import numpy as np
    d, k = zmc.make_desc(1, 2, [0, 0], [1, 1], [20, 20], np.linspace(0.5, 5, 40), 1 << 14, 4, 0)
    r = zmc.zmc_autotune(d, 200)
    print(json.dumps([r.lanes, r.block, r.groups_per_lane]))
else:
    r = zmc.zmc_autotune_lookup(2, 1, 2, 1 << 14)
    print(json.dumps(None if r is None else [r.lanes, r.block, r.groups_per_lane]))
""" % ROOT


def test_cache_file_round_trip(tmp_path):
    pytest.importorskip("torch")
    env = dict(os.environ, ZMC_AUTOTUNE_CACHE=str(tmp_path / "tune.txt"))
    a = subprocess.run([sys.executable, "-c", CHILD, "tune"], env=env, capture_output=True,
                       text=True, timeout=600)
    assert a.returncode == 0, a.stderr[-2000:]
    b = subprocess.run([sys.executable, "-c", CHILD, "lookup"], env=env, capture_output=True,
                       text=True, timeout=600)
    assert b.returncode == 0, b.stderr[-2000:]
    assert json.loads(a.stdout.strip().splitlines()[-1]) == \
        json.loads(b.stdout.strip().splitlines()[-1])
