"""Philox4x32-10 against cuRAND's device implementation (a third party).

Pins both the oracle's Philox (CPU) and the library's hoisted device Philox
(through zmc_stream_words) to curand_Philox4x32_10 on the same counters.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand") / "libprobe.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", "-o", out, os.path.join(HERE, "curand_probe.cu")],
                   check=True)
    lib = ctypes.CDLL(out)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.curand_probe_philox.argtypes = [u32p, u32p, ctypes.c_int, u32p]
    lib.curand_probe_philox.restype = ctypes.c_int
    return lib


def _curand(lib, ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros((len(c), 4), dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = lib.curand_probe_philox(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), len(c),
                                 out.ctypes.data_as(u32p))
    assert rc == 0
    return out


def test_oracle_philox_matches_curand(probe):
    rng = np.random.default_rng(77)
    ctr = rng.integers(0, 2 ** 32, (500, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (500, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    ref = _curand(probe, ctr, key)
    O = oracle.default()
    for i in range(len(ctr)):
        assert O.philox4x32_10(ctr[i], key[i]) == [int(v) for v in ref[i]], i


def test_library_stream_matches_curand(probe):
    from paper_1910_01965_gb300 import zmc
    for seed, p, t in [(0, 0, 0), (2 ** 64 - 1, 2 ** 61 + 7, 2 ** 31 - 1), (99, 123456789, 3)]:
        n = 4 * 300
        words = zmc.zmc_stream_words(seed, p, t, 0, n)
        ctr = np.array([[j, t, p & 0xFFFFFFFF, p >> 32] for j in range(n // 4)],
                       dtype=np.uint64).astype(np.uint32)
        key = np.array([[seed & 0xFFFFFFFF, seed >> 32]] * (n // 4),
                       dtype=np.uint64).astype(np.uint32)
        ref = _curand(probe, ctr, key).reshape(-1)
        assert np.array_equal(words, ref), (seed, p, t)
