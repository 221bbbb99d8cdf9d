"""Long scans in slices of the flat grid, checkpointed to disk and resumable.

The paper targets grids of up to 1e10 points (Abstract, Sec. 1) cut into
batches (Sec. 2).  Here a scan is evaluated slice by slice through the slice
API (first_index, count); every finished slice's results go into .npy files
opened as memory maps, and a small JSON progress file records the number of
finished slices (written atomically after the data is flushed).  A scan that
is interrupted resumes at the first unfinished slice.  Every sample's random
stream is keyed by the global flat index, and the tile configuration is
pinned for the whole scan, so the results are bit-identical to one
uninterrupted whole-grid scan with the same tiles.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Optional, Sequence

import numpy as np

FIELDS = ("mean", "err", "errw")


class CheckpointedScan:
    """One scan of P grid points in slices of `slice_points`, stored under `path`.

    `scan_fn(first_index, count, tiles)` evaluates one slice and returns a dict
    of arrays (mean, err, errw) of `count` entries each and the tile
    configuration it used; `tiles` is the pinned (lanes, splits, block).  The
    default uses the library's zmc_scan_ex with host buffers.
    """

    def __init__(self, path: str, P: int, slice_points: int,
                 scan_fn: Callable[[int, int, Sequence[int]], dict],
                 tiles: Sequence[int], meta: Optional[dict] = None):
        if P < 1 or slice_points < 1:
            raise ValueError("P and slice_points must be positive")
        self.path = path
        self.P = int(P)
        self.slice_points = int(slice_points)
        self.nslices = (self.P + self.slice_points - 1) // self.slice_points
        self.scan_fn = scan_fn
        self.tiles = tuple(int(t) for t in tiles)
        os.makedirs(path, exist_ok=True)
        self.progress_file = os.path.join(path, "progress.json")
        state = self._read_progress()
        want = {"P": self.P, "slice_points": self.slice_points, "tiles": list(self.tiles),
                "meta": meta or {}}
        if state is None:
            self.done = 0
            for f in FIELDS:
                np.lib.format.open_memmap(self._file(f), mode="w+", dtype=np.float64,
                                          shape=(self.P,))
            self._write_progress(want)
        else:
            for k in ("P", "slice_points", "tiles", "meta"):
                if state.get(k) != want[k]:
                    raise ValueError("checkpoint at %s was made for another scan (%s differs)"
                                     % (path, k))
            self.done = int(state["done"])

    def _file(self, field):
        return os.path.join(self.path, field + ".npy")

    def _read_progress(self):
        if not os.path.exists(self.progress_file):
            return None
        with open(self.progress_file) as f:
            return json.load(f)

    def _write_progress(self, base):
        tmp = self.progress_file + ".tmp"
        with open(tmp, "w") as f:
            json.dump(dict(base, done=self.done, nslices=self.nslices), f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self.progress_file)

    @property
    def finished(self) -> bool:
        return self.done >= self.nslices

    def run(self, max_slices: Optional[int] = None) -> bool:
        """Evaluate unfinished slices (at most `max_slices`); True when the
        whole scan is on disk."""
        base = self._read_progress()
        todo = self.nslices - self.done if max_slices is None else min(
            max_slices, self.nslices - self.done)
        maps = {f: np.load(self._file(f), mmap_mode="r+") for f in FIELDS}
        for _ in range(todo):
            first = self.done * self.slice_points
            count = min(self.slice_points, self.P - first)
            res = self.scan_fn(first, count, self.tiles)
            for f in FIELDS:
                maps[f][first:first + count] = res[f]
                maps[f].flush()
            self.done += 1
            self._write_progress(base)
        return self.finished

    def results(self) -> dict:
        return {f: np.load(self._file(f), mmap_mode="r") for f in FIELDS}


def library_scan_fn(gid, N, lo, hi, lengths, values, S, T, seed, precision=2):
    """scan_fn over zmc_scan_ex (host buffers) for CheckpointedScan."""
    from . import zmc

    def fn(first, count, tiles):
        res, o = zmc.scan(gid, N, lo, hi, lengths, values, S, T, seed, precision=precision,
                          first_index=first, count=count, tiles=tiles)
        return res
    return fn


def planned_tiles(gid, N, lo, hi, lengths, values, S, T, seed, precision=2):
    """The tile configuration the planner picks for the whole grid (planned
    with ZMC_F_PLAN_ONLY, nothing is computed)."""
    from . import zmc
    d, keep = zmc.make_desc(gid, N, lo, hi, lengths, values, S, T, seed, precision,
                            flags=zmc.ZMC_F_PLAN_ONLY)
    o = zmc.zmc_scan_out()
    zmc.zmc_scan_ex(d, o)
    return (o.tile_lanes, o.tile_splits, o.tile_block)
