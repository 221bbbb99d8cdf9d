"""Slice-by-slice checkpointing: bookkeeping on the CPU with a stand-in scan."""
import json

import numpy as np
import pytest

from paper_1910_01965_gb300.checkpoint import CheckpointedScan


def fake_scan(first, count, tiles):
    idx = np.arange(first, first + count, dtype=np.float64)
    return {"mean": idx * 2.0 + tiles[0], "err": idx + 0.5, "errw": -idx}


def test_resume_after_interruption_gives_the_uninterrupted_result(tmp_path):
    P, sl, tiles = 1003, 100, (8, 2, 256)
    a = CheckpointedScan(str(tmp_path / "a"), P, sl, fake_scan, tiles)
    assert not a.run(max_slices=3)
    assert json.load(open(tmp_path / "a" / "progress.json"))["done"] == 3
    b = CheckpointedScan(str(tmp_path / "a"), P, sl, fake_scan, tiles)  # a new process
    assert b.done == 3 and b.run()
    whole = CheckpointedScan(str(tmp_path / "w"), P, sl, fake_scan, tiles)
    assert whole.run()
    for f in ("mean", "err", "errw"):
        assert np.array_equal(b.results()[f], whole.results()[f])
    assert np.array_equal(b.results()["mean"], np.arange(P) * 2.0 + 8)


def test_a_failed_slice_is_redone_not_skipped(tmp_path):
    P, sl, tiles = 500, 64, (4, 1, 128)
    calls = []

    def flaky(first, count, t):
        calls.append(first)
        if len(calls) == 4:
            raise RuntimeError("device lost")
        return fake_scan(first, count, t)

    c = CheckpointedScan(str(tmp_path / "c"), P, sl, flaky, tiles)
    with pytest.raises(RuntimeError):
        c.run()
    assert c.done == 3
    c2 = CheckpointedScan(str(tmp_path / "c"), P, sl, fake_scan, tiles)
    assert c2.run()
    assert np.array_equal(c2.results()["err"], np.arange(P) + 0.5)


def test_checkpoint_of_another_scan_is_refused(tmp_path):
    CheckpointedScan(str(tmp_path / "d"), 100, 10, fake_scan, (8, 1, 256)).run(max_slices=1)
    with pytest.raises(ValueError):
        CheckpointedScan(str(tmp_path / "d"), 100, 10, fake_scan, (16, 1, 256))
    with pytest.raises(ValueError):
        CheckpointedScan(str(tmp_path / "d"), 101, 10, fake_scan, (8, 1, 256))
