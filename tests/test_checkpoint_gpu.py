"""A checkpointed scan, interrupted and resumed, equals one whole-grid scan
bit for bit (same pinned tiles)."""
import numpy as np
import pytest

from paper_1910_01965_gb300 import checkpoint as ck
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_interrupted_and_resumed_scan_is_bit_identical(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc
    spec = wl.scan_osc_1e4(samples=1 << 12, trials=3)
    args = (spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
            spec.samples, spec.trials, spec.seed)
    tiles = ck.planned_tiles(*args)
    fn = ck.library_scan_fn(*args)
    a = ck.CheckpointedScan(str(tmp_path / "s"), spec.P, 1500, fn, tiles)
    assert not a.run(max_slices=2)
    b = ck.CheckpointedScan(str(tmp_path / "s"), spec.P, 1500, fn, tiles)
    assert b.done == 2 and b.run()
    whole, o = zmc.scan(*args, tiles=tiles)
    for f in ("mean", "err", "errw"):
        assert np.array_equal(np.asarray(b.results()[f]), whole[f])
