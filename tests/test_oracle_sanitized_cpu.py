"""The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer.

The FP64 CPU oracle (oracle/zmc_oracle.c) is compiled a second time with
-fsanitize=address,undefined (no recovery: the first report aborts) and run
in a child process on small scans of every integrand at N = 1..8, including
grid indices beyond 2^32; any out-of-bounds access, overflow or other
undefined behaviour fails the test, and the results must equal the regular
build's bit for bit (the same FP64 arithmetic in the same order).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(here)r)
from oracle import oracle
import test_oracle_sanitized_cpu as t
O = oracle.Oracle(sys.argv[1])
np.save(sys.argv[2], t.run_cases(O))
"""


def _cases():
    r = np.random.default_rng(23)
    out = []
    for N in range(1, 9):
        lens = ([3, 2, 2] + [1] * 5)[:N]
        for gid in range(6):
            if gid in (oracle.G_CONST, oracle.G_SINSUM):
                lists, lo, hi = [np.arange(4.0), np.arange(3.0)], np.zeros(N), 2 * np.ones(N)
            elif gid == oracle.G_GAUSS03:
                lists, lo, hi = [r.uniform(-1, 1, k) for k in lens], -np.ones(N), np.ones(N)
            else:
                lists, lo, hi = [r.uniform(0.5, 5, k) for k in lens], np.zeros(N), np.ones(N)
            out.append((gid, N, lo, hi, lists, int(r.integers(1, 65)), int(r.integers(1, 4)),
                        int(r.integers(0, 2 ** 63))))
    return out


def run_cases(O):
    """Every case's mean, err and errw, then sampled points of a grid beyond
    2^32 points, concatenated into one array."""
    parts = []
    for gid, N, lo, hi, lists, S, T, seed in _cases():
        lens = np.array([len(v) for v in lists], np.int64)
        res = O.scan(gid, N, lo, hi, lens, np.concatenate(lists), S, T, seed)
        parts += [res["mean"], res["err"], res["errw"]]
    big = [np.linspace(0.5, 5, 2048), np.linspace(0.5, 5, 2048), np.linspace(0.5, 5, 1025)]
    lens = np.array([len(v) for v in big], np.int64)
    pts = np.array([0, (1 << 32) - 1, 1 << 32, (1 << 32) + 12345, int(np.prod(lens)) - 1],
                   np.int64)
    res = O.scan_points(oracle.G_COSPROD, 3, np.zeros(3), np.ones(3), lens,
                        np.concatenate(big), 40, 2, 99, pts)
    parts += [res["mean"], res["err"]]
    return np.concatenate(parts)


def test_sanitized_oracle_runs_clean_and_matches(tmp_path):
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                          text=True).stdout.strip()
    if not asan or not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("gcc's AddressSanitizer runtime is not installed")
    lib = str(tmp_path / "libzmc_oracle_san.so")
    flags = [f for f in oracle.CFLAGS if f != "-O2"] + [
        "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
        "-fno-sanitize-recover=all"]
    subprocess.run(["gcc", *flags, "-o", lib, oracle.SOURCE, "-lm"], check=True)
    out = str(tmp_path / "san.npy")
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT, "here": HERE}, lib, out],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
    got = np.load(out)
    ref = run_cases(oracle.default())
    assert got.shape == ref.shape
    assert np.array_equal(got, ref, equal_nan=True)
