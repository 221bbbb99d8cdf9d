"""Python wrapper of the FP64 CPU oracle (zmc_oracle.c).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  The CUDA product path never imports it.
It imports nothing from the product package, and the product package imports
nothing from here.

The oracle is the direct Monte Carlo estimator of Eq. 1 (Sec. 2) over a
Cartesian parameter grid, written out in FP64 in plain sequential order; the
random stream is Philox4x32-10 (SC'11) with the counter layout documented in
zmc_oracle.c.  ``build()`` compiles it with gcc; nothing here runs on a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "zmc_oracle.c")
LIBRARY = os.path.join(_HERE, "libzmc_oracle.so")

# Registry ids, equal in value (not shared in code) to the library's table.
G_CONST, G_COSPROD, G_GAUSS03, G_POLY, G_OSC01, G_SINSUM = range(6)
G_NAMES = ["const", "cosprod", "gauss03", "poly", "osc01", "sinsum"]

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-fopenmp", "-fPIC", "-shared", "-Wall"]


def compile_source(src: str, out: str) -> str:
    """gcc-compile an oracle source file into a shared library."""
    tmp = out + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libzmc_oracle.so (gcc, OpenMP, -O2)."""
    if (not force and os.path.exists(LIBRARY)
            and os.path.getmtime(LIBRARY) >= os.path.getmtime(SOURCE)):
        return LIBRARY
    return compile_source(SOURCE, LIBRARY)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class Oracle:
    """One loaded build of the oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.zmc_oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.zmc_oracle_philox4x32_10.restype = None
        lib.zmc_oracle_uniform.argtypes = [ctypes.c_uint32]
        lib.zmc_oracle_uniform.restype = ctypes.c_double
        lib.zmc_oracle_word.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_int, ctypes.c_uint64]
        lib.zmc_oracle_word.restype = ctypes.c_uint32
        lib.zmc_oracle_field.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_uint64]
        lib.zmc_oracle_field.restype = ctypes.c_uint32
        lib.zmc_oracle_sample_y.argtypes = [ctypes.c_int, dp, dp,
                                            ctypes.c_uint64, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_int64, dp]
        lib.zmc_oracle_sample_y.restype = None
        lib.zmc_oracle_decode.argtypes = [ctypes.c_int, i64p, ctypes.c_int64,
                                          i64p]
        lib.zmc_oracle_decode.restype = None
        lib.zmc_oracle_grid_point.argtypes = [ctypes.c_int, i64p, dp,
                                              ctypes.c_int64, dp]
        lib.zmc_oracle_grid_point.restype = None
        lib.zmc_oracle_integrand_valid.argtypes = [ctypes.c_int] * 3
        lib.zmc_oracle_integrand_valid.restype = ctypes.c_int
        lib.zmc_oracle_integrand.argtypes = [ctypes.c_int, ctypes.c_int, dp,
                                             ctypes.c_int, dp]
        lib.zmc_oracle_integrand.restype = ctypes.c_double
        lib.zmc_oracle_scan_points.argtypes = [
            ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, i64p, dp,
            ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, i64p,
            ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_int]
        lib.zmc_oracle_scan_points.restype = ctypes.c_int
        lib.zmc_oracle_max_threads.argtypes = []
        lib.zmc_oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    # -- building blocks ---------------------------------------------------
    def philox4x32_10(self, ctr, key):
        """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
        c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
        k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
        o = (ctypes.c_uint32 * 4)()
        self.lib.zmc_oracle_philox4x32_10(c, k, o)
        return [int(v) for v in o]

    def uniform(self, v: int) -> float:
        """u = (2 v + 1) 2^-24 for a 23-bit field value v."""
        return self.lib.zmc_oracle_uniform(int(v) & 0xFFFFFFFF)

    def word(self, seed: int, p: int, t: int, w: int) -> int:
        """Raw word w of the Philox stream of (seed, p, t)."""
        return int(self.lib.zmc_oracle_word(seed, p, t, w))

    def field(self, seed: int, p: int, t: int, i: int) -> int:
        """23-bit field i of the stream of (seed, p, t)."""
        return int(self.lib.zmc_oracle_field(seed, p, t, i))

    def sample_y(self, N, lo, hi, seed, p, t, s):
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        y = np.zeros(N, dtype=np.float64)
        self.lib.zmc_oracle_sample_y(N, _dp(lo), _dp(hi), seed, p, t, s, _dp(y))
        return y

    def decode(self, lengths, p):
        lengths = np.ascontiguousarray(lengths, dtype=np.int64)
        d = np.zeros(len(lengths), dtype=np.int64)
        self.lib.zmc_oracle_decode(len(lengths), _i64p(lengths), int(p), _i64p(d))
        return d

    def grid_point(self, lengths, values, p):
        lengths = np.ascontiguousarray(lengths, dtype=np.int64)
        values = np.ascontiguousarray(values, dtype=np.float64)
        x = np.zeros(len(lengths), dtype=np.float64)
        self.lib.zmc_oracle_grid_point(len(lengths), _i64p(lengths),
                                       _dp(values), int(p), _dp(x))
        return x

    def integrand(self, gid, y, x):
        y = np.ascontiguousarray(y, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        return self.lib.zmc_oracle_integrand(gid, len(y), _dp(y), len(x), _dp(x))

    def integrand_valid(self, gid, N, M) -> bool:
        return bool(self.lib.zmc_oracle_integrand_valid(gid, N, M))

    def max_threads(self) -> int:
        return int(self.lib.zmc_oracle_max_threads())

    # -- the estimator -----------------------------------------------------
    def scan_points(self, gid, N, lo, hi, lengths, values, S, T, seed, points,
                    want_sums=False, nthreads=0):
        """Oracle estimates at the flat grid indices ``points``.

        Returns a dict with ``mean``, ``err``, ``errw`` (each [npoints]) and,
        with ``want_sums``, ``s1`` and ``s2`` ([npoints, T]).  Raises
        ValueError when the oracle rejects the arguments.
        """
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        lengths = np.ascontiguousarray(lengths, dtype=np.int64)
        values = np.ascontiguousarray(values, dtype=np.float64)
        points = np.ascontiguousarray(points, dtype=np.int64)
        n = points.size
        mean, err, errw = np.zeros(n), np.zeros(n), np.zeros(n)
        s1 = np.zeros((n, T)) if want_sums else None
        s2 = np.zeros((n, T)) if want_sums else None
        null = ctypes.POINTER(ctypes.c_double)()
        rc = self.lib.zmc_oracle_scan_points(
            int(gid), int(N), _dp(lo), _dp(hi), len(lengths), _i64p(lengths),
            _dp(values), int(S), int(T), int(seed), _i64p(points), n,
            _dp(mean), _dp(err), _dp(errw),
            _dp(s1) if want_sums else null, _dp(s2) if want_sums else null,
            int(nthreads))
        if rc != 0:
            raise ValueError("oracle rejected the arguments (status %d)" % rc)
        out = {"mean": mean, "err": err, "errw": errw}
        if want_sums:
            out["s1"], out["s2"] = s1, s2
        return out

    def scan(self, gid, N, lo, hi, lengths, values, S, T, seed,
             want_sums=False, nthreads=0):
        """Oracle estimates at every grid point, in C order over the lists."""
        P = int(np.prod(np.asarray(lengths, dtype=np.int64)))
        return self.scan_points(gid, N, lo, hi, lengths, values, S, T, seed,
                                np.arange(P, dtype=np.int64), want_sums,
                                nthreads)


_lock = threading.Lock()
_default = None


def default() -> Oracle:
    """The oracle built from oracle/zmc_oracle.c (compiled on first use)."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
        return _default


def scan(*args, **kwargs):
    return default().scan(*args, **kwargs)


def scan_points(*args, **kwargs):
    return default().scan_points(*args, **kwargs)
