"""Thin ctypes binding of the C ABI in include/zmc.h (libzmc.so).

Argument marshalling only: every step of a scan runs in the library's CUDA
kernels.  The names mirror the C entry points (``zmc_scan``, ``zmc_scan_ex``,
...).  ``scan()`` and ``scan_device()`` are conveniences that fill a
``zmc_scan_desc`` from numpy arrays or torch CUDA tensors and call
``zmc_scan_ex``.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# ZMC_LIBRARY names another build of the library (e.g. libzmc_debug.so).
LIBRARY = os.environ.get("ZMC_LIBRARY") or os.path.join(_PKG, "libzmc.so")

ZMC_OK, ZMC_EINVAL, ZMC_ENOMEM, ZMC_ECUDA, ZMC_ETIMEDOUT, ZMC_ECANCELED, \
    ZMC_EBUSY, ZMC_ENOTFOUND = range(8)
ZMC_FP64, ZMC_FP32, ZMC_FP32_KAHAN = range(3)
ZMC_G_CONST, ZMC_G_COSPROD, ZMC_G_GAUSS03, ZMC_G_POLY, ZMC_G_OSC01, \
    ZMC_G_SINSUM, ZMC_G_COUNT = range(7)
ZMC_MEM_HOST, ZMC_MEM_DEVICE = 0, 1
ZMC_F_TIMINGS, ZMC_F_SYNC, ZMC_F_PLAN_ONLY = 1, 2, 4
ZMC_MAX_N, ZMC_MAX_M = 8, 16

STATUS_NAMES = {0: "ZMC_OK", 1: "ZMC_EINVAL", 2: "ZMC_ENOMEM", 3: "ZMC_ECUDA",
                4: "ZMC_ETIMEDOUT", 5: "ZMC_ECANCELED", 6: "ZMC_EBUSY",
                7: "ZMC_ENOTFOUND"}
PRECISIONS = {"fp64": ZMC_FP64, "fp32": ZMC_FP32, "fp32_kahan": ZMC_FP32_KAHAN}


class ZmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


class zmc_scan_desc(ctypes.Structure):
    _fields_ = [("integrand_id", ctypes.c_int), ("N", ctypes.c_int),
                ("lo", _dp), ("hi", _dp), ("M", ctypes.c_int),
                ("list_len", _i64p), ("list_vals", _dp),
                ("samples_per_point", ctypes.c_int64), ("trials", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int),
                ("mem", ctypes.c_int), ("first_index", ctypes.c_int64),
                ("count", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("tile_lanes", ctypes.c_int), ("tile_splits", ctypes.c_int),
                ("tile_block", ctypes.c_int), ("flags", ctypes.c_int),
                ("chunk_points", ctypes.c_int64)]


class zmc_scan_out(ctypes.Structure):
    _fields_ = [("mean", _dp), ("err", _dp), ("errw", _dp), ("s1", _dp), ("s2", _dp),
                ("tile_lanes", ctypes.c_int), ("tile_splits", ctypes.c_int),
                ("tile_block", ctypes.c_int), ("launches", ctypes.c_int),
                ("h2d_ms", ctypes.c_float), ("kernel_ms", ctypes.c_float),
                ("finalize_ms", ctypes.c_float), ("d2h_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("chunks", ctypes.c_int64)]


class zmc_integrand_info(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int), ("name", ctypes.c_char * 32),
                ("m_rule", ctypes.c_int)]


class zmc_device_info(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("sm_count", ctypes.c_int),
                ("cc_major", ctypes.c_int), ("cc_minor", ctypes.c_int),
                ("max_threads_per_sm", ctypes.c_int), ("clock_khz", ctypes.c_int),
                ("total_mem", ctypes.c_size_t), ("name", ctypes.c_char * 96)]


class zmc_pipe_result(ctypes.Structure):
    _fields_ = [("pipe", ctypes.c_int), ("ops_per_clk_per_sm", ctypes.c_double),
                ("ops_per_s", ctypes.c_double), ("clock_mhz", ctypes.c_double),
                ("ms", ctypes.c_double), ("ops", ctypes.c_int64)]


class zmc_batch_info(ctypes.Structure):
    _fields_ = [("scans", ctypes.c_int), ("precisions", ctypes.c_int),
                ("tiles", ctypes.c_int64), ("evaluations", ctypes.c_int64),
                ("grid", ctypes.c_int), ("block", ctypes.c_int),
                ("scratch_bytes", ctypes.c_size_t), ("graph", ctypes.c_int),
                ("launches_per_run", ctypes.c_int)]


ZMC_BATCH_GRAPH = 1


class zmc_server_opts(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("step_ms", ctypes.c_double),
                ("chunk_units", ctypes.c_int64), ("fail_alloc_every", ctypes.c_int)]


class zmc_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("active", ctypes.c_int64),
                ("max_queued", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("evaluations", ctypes.c_int64), ("busy_ms", ctypes.c_double),
                ("evals_per_s", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mem_in_use", ctypes.c_size_t),
                ("mem_peak", ctypes.c_size_t)]

class zmc_tune_result(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int), ("block", ctypes.c_int),
                ("groups_per_lane", ctypes.c_int), ("candidates", ctypes.c_int),
                ("evals_per_s", ctypes.c_double), ("default_evals_per_s", ctypes.c_double)]


PIPE_NAMES = ["FFMA", "IMAD", "IMAD.WIDE", "IMAD.HI", "LOP3", "SHF", "MUFU.RSQ",
              "MUFU.EX2+LG2", "DFMA", "PHILOX_CALL", "MUFU.EX2", "MUFU.COS", "FFMA2",
              "IMAD.WIDE+2FFMA", "IMAD.WIDE+FFMA2"]

# (name, restype, argtypes) of every exported entry point this binding uses.
SIGNATURES = [
    ("zmc_version", ctypes.c_int, []),
    ("zmc_last_error", ctypes.c_char_p, []),
    ("zmc_scan_desc_init", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc)]),
    ("zmc_integrand_info_get", ctypes.c_int, [ctypes.c_int,
                                              ctypes.POINTER(zmc_integrand_info)]),
    ("zmc_device_info_get", ctypes.c_int, [ctypes.POINTER(zmc_device_info)]),
    ("zmc_validate", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc)]),
    ("zmc_workspace_size", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    ("zmc_scan", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                _i64p, _dp, ctypes.c_int64, ctypes.c_int,
                                ctypes.c_uint64, _dp, _dp]),
    ("zmc_scan_ex", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc),
                                   ctypes.POINTER(zmc_scan_out)]),
    ("zmc_stream_words", ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_uint32)]),
    ("zmc_pipe_measure", ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(zmc_pipe_result)]),
    ("zmc_scan_noalloc", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc),
                                        ctypes.POINTER(zmc_scan_out)]),
    ("zmc_batch_create", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc),
                                        ctypes.POINTER(zmc_scan_out), ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("zmc_batch_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("zmc_batch_info_get", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(zmc_batch_info)]),
    ("zmc_batch_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("zmc_scan_batch", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc), ctypes.c_int,
                                      ctypes.POINTER(zmc_scan_out)]),
    ("zmc_server_opts_init", ctypes.c_int, [ctypes.POINTER(zmc_server_opts)]),
    ("zmc_server_create", ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(zmc_server_opts),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    ("zmc_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(zmc_scan_desc),
                                  ctypes.POINTER(zmc_scan_out),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    ("zmc_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                ctypes.POINTER(ctypes.c_int)]),
    ("zmc_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]),
    ("zmc_cancel", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("zmc_server_stats_get", ctypes.c_int, [ctypes.c_void_p,
                                            ctypes.POINTER(zmc_server_stats)]),
    ("zmc_server_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("zmc_autotune", ctypes.c_int, [ctypes.POINTER(zmc_scan_desc), ctypes.c_int,
                                    ctypes.POINTER(zmc_tune_result)]),
    ("zmc_autotune_lookup", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int64, ctypes.POINTER(zmc_tune_result)]),
    ("zmc_autotune_reset", ctypes.c_int, []),
    ("zmc_integrand_register", ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int,
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("zmc_debug_failures", ctypes.c_int64, [ctypes.POINTER(ctypes.c_uint),
                                            ctypes.POINTER(ctypes.c_longlong)]),
]

_lock = threading.Lock()
_lib = None


def load(path: str = LIBRARY):
    """Load libzmc.so (built by __graft_entry__.build()); raise if missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                "libzmc.so is not built (%s); run __graft_entry__.build() — "
                "there is no CPU fallback" % path)
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != ZMC_OK:
        raise ZmcError(rc, load().zmc_last_error().decode(errors="replace"))


# ------------------------------------------------------- same-name wrappers --
def zmc_version() -> int:
    return load().zmc_version()


def zmc_last_error() -> str:
    return load().zmc_last_error().decode(errors="replace")


def zmc_debug_failures():
    """(failed device-side checks since the last call, first failure's code,
    its index); failures = -1 in builds without checks."""
    code, index = ctypes.c_uint(0), ctypes.c_longlong(0)
    n = load().zmc_debug_failures(ctypes.byref(code), ctypes.byref(index))
    return int(n), int(code.value), int(index.value)


def zmc_scan_desc_init() -> zmc_scan_desc:
    d = zmc_scan_desc()
    _check(load().zmc_scan_desc_init(ctypes.byref(d)))
    return d


def zmc_integrand_info_get(gid: int) -> zmc_integrand_info:
    info = zmc_integrand_info()
    _check(load().zmc_integrand_info_get(gid, ctypes.byref(info)))
    return info


def zmc_device_info_get() -> zmc_device_info:
    info = zmc_device_info()
    _check(load().zmc_device_info_get(ctypes.byref(info)))
    return info


def zmc_validate(d: zmc_scan_desc) -> int:
    return load().zmc_validate(ctypes.byref(d))


def zmc_workspace_size(d: zmc_scan_desc) -> int:
    n = ctypes.c_size_t(0)
    _check(load().zmc_workspace_size(ctypes.byref(d), ctypes.byref(n)))
    return int(n.value)


def zmc_scan(gid, N, lo, hi, lengths, values, S, T, seed):
    """The simple host entry point; returns (mean, err) numpy arrays."""
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    L = np.ascontiguousarray(lengths, np.int64)
    v = np.ascontiguousarray(values, np.float64)
    P = int(np.prod(L))
    mean = np.empty(P)
    err = np.empty(P)
    _check(load().zmc_scan(int(gid), int(N), lo.ctypes.data_as(_dp), hi.ctypes.data_as(_dp),
                           len(L), L.ctypes.data_as(_i64p), v.ctypes.data_as(_dp),
                           int(S), int(T), int(seed), mean.ctypes.data_as(_dp),
                           err.ctypes.data_as(_dp)))
    return mean, err


def zmc_scan_ex(d: zmc_scan_desc, o: zmc_scan_out) -> zmc_scan_out:
    _check(load().zmc_scan_ex(ctypes.byref(d), ctypes.byref(o)))
    return o


def zmc_stream_words(seed: int, p: int, t: int, first_word: int, nwords: int) -> np.ndarray:
    out = np.zeros(nwords, dtype=np.uint32)
    _check(load().zmc_stream_words(int(seed), int(p), int(t), int(first_word), int(nwords),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return out


def zmc_pipe_measure(pipe: int, iterations: int = 4096) -> zmc_pipe_result:
    r = zmc_pipe_result()
    _check(load().zmc_pipe_measure(int(pipe), int(iterations), ctypes.byref(r)))
    return r


ZMC_NOALLOC_SCRATCH_BYTES = 16 << 20


def zmc_scan_noalloc(d: zmc_scan_desc, o: zmc_scan_out) -> zmc_scan_out:
    """The scan entry point that allocates nothing (device-memory lists and
    outputs; scratch is the library's fixed 16 MiB device array)."""
    _check(load().zmc_scan_noalloc(ctypes.byref(d), ctypes.byref(o)))
    return o


def zmc_batch_create(descs, outs, flags=0):
    """descs, outs: ctypes arrays (or lists) of zmc_scan_desc / zmc_scan_out.
    Returns the opaque batch handle (int)."""
    n = len(descs)
    D = (zmc_scan_desc * n)(*descs)
    O = (zmc_scan_out * n)(*outs)
    h = ctypes.c_void_p()
    _check(load().zmc_batch_create(D, O, n, int(flags), ctypes.byref(h)))
    for i in range(n):
        outs[i].tile_lanes, outs[i].tile_splits = O[i].tile_lanes, O[i].tile_splits
        outs[i].tile_block = O[i].tile_block
    return h.value


def zmc_batch_run(handle, stream=None):
    _check(load().zmc_batch_run(ctypes.c_void_p(handle), stream))


def zmc_batch_info_get(handle) -> zmc_batch_info:
    info = zmc_batch_info()
    _check(load().zmc_batch_info_get(ctypes.c_void_p(handle), ctypes.byref(info)))
    return info


def zmc_batch_destroy(handle):
    _check(load().zmc_batch_destroy(ctypes.c_void_p(handle)))


def zmc_scan_batch(descs, outs):
    n = len(descs)
    D = (zmc_scan_desc * n)(*descs)
    O = (zmc_scan_out * n)(*outs)
    _check(load().zmc_scan_batch(D, n, O))
    for i in range(n):
        outs[i] = O[i]
    return outs


def zmc_server_opts_init() -> zmc_server_opts:
    o = zmc_server_opts()
    _check(load().zmc_server_opts_init(ctypes.byref(o)))
    return o


def zmc_server_create(budget_bytes: int, opts: zmc_server_opts = None) -> int:
    h = ctypes.c_void_p()
    _check(load().zmc_server_create(int(budget_bytes),
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(h)))
    return h.value


def zmc_submit(server: int, d: zmc_scan_desc, o: zmc_scan_out) -> int:
    t = ctypes.c_uint64()
    _check(load().zmc_submit(ctypes.c_void_p(server), ctypes.byref(d), ctypes.byref(o),
                             ctypes.byref(t)))
    return int(t.value)


def zmc_poll(server: int, ticket: int) -> bool:
    done = ctypes.c_int()
    _check(load().zmc_poll(ctypes.c_void_p(server), int(ticket), ctypes.byref(done)))
    return bool(done.value)


def zmc_wait(server: int, ticket: int, timeout_ms: int = -1) -> int:
    """Returns the request's final status code (ZMC_OK, ZMC_ECANCELED, ...)
    or ZMC_ETIMEDOUT; raises only for an unknown ticket."""
    rc = load().zmc_wait(ctypes.c_void_p(server), int(ticket), int(timeout_ms))
    if rc == ZMC_ENOTFOUND:
        _check(rc)
    return rc


def zmc_cancel(server: int, ticket: int) -> int:
    return load().zmc_cancel(ctypes.c_void_p(server), int(ticket))


def zmc_server_stats_get(server: int) -> zmc_server_stats:
    st = zmc_server_stats()
    _check(load().zmc_server_stats_get(ctypes.c_void_p(server), ctypes.byref(st)))
    return st


def zmc_server_destroy(server: int):
    _check(load().zmc_server_destroy(ctypes.c_void_p(server)))


def zmc_autotune(d: zmc_scan_desc, budget_ms: int = 500) -> zmc_tune_result:
    r = zmc_tune_result()
    _check(load().zmc_autotune(ctypes.byref(d), int(budget_ms), ctypes.byref(r)))
    return r


def zmc_autotune_lookup(precision, gid, N, samples):
    r = zmc_tune_result()
    rc = load().zmc_autotune_lookup(int(precision), int(gid), int(N), int(samples),
                                    ctypes.byref(r))
    if rc == ZMC_ENOTFOUND:
        return None
    _check(rc)
    return r


def zmc_autotune_reset():
    _check(load().zmc_autotune_reset())


ZMC_G_USER_BASE = 1000


def zmc_integrand_register(name: str, source: str, n_min: int = 1, n_max: int = ZMC_MAX_N):
    """Compile a user integrand (CUDA C source defining zmc_user_g32 and/or
    zmc_user_g64) with NVRTC; returns its integrand id."""
    i = ctypes.c_int()
    _check(load().zmc_integrand_register(name.encode(), source.encode(), int(n_min),
                                         int(n_max), ctypes.byref(i)))
    return int(i.value)


class Server:
    """Keeps each request's descriptor and host output arrays alive until the
    caller has collected them (marshalling only; the loop is the library's)."""

    def __init__(self, budget_bytes: int, **opts):
        o = zmc_server_opts_init()
        for k, v in opts.items():
            setattr(o, k, v)
        self.handle = zmc_server_create(budget_bytes, o)
        self.requests = {}

    def submit(self, gid, N, lo, hi, lengths, values, S, T, seed, precision=ZMC_FP32_KAHAN,
               first_index=0, count=-1, tiles=(0, 0, 0), want_sums=False):
        d, keep = make_desc(gid, N, lo, hi, lengths, values, S, T, seed, precision,
                            ZMC_MEM_HOST, first_index, count, None, tiles)
        P = int(np.prod(np.asarray(lengths, np.int64)))
        n = (P - first_index) if count < 0 else count
        res = {"mean": np.empty(n), "err": np.empty(n), "errw": np.empty(n)}
        if want_sums:
            res["s1"] = np.empty((n, T))
            res["s2"] = np.empty((n, T))
        o = zmc_scan_out()
        o.mean, o.err, o.errw = _ptr(res["mean"]), _ptr(res["err"]), _ptr(res["errw"])
        o.s1, o.s2 = _ptr(res.get("s1")), _ptr(res.get("s2"))
        t = zmc_submit(self.handle, d, o)
        self.requests[t] = (d, o, res, keep)
        return t

    def wait(self, ticket, timeout_ms=-1):
        return zmc_wait(self.handle, ticket, timeout_ms)

    def result(self, ticket):
        d, o, res, keep = self.requests[ticket]
        return res, o

    def stats(self):
        return zmc_server_stats_get(self.handle)

    def close(self):
        if self.handle:
            zmc_server_destroy(self.handle)
            self.handle = None


# -------------------------------------------------------------- helpers --
class _Keep:
    """Holds numpy buffers alive while a descriptor points into them."""

    def __init__(self):
        self.items = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype)
        self.items.append(a)
        return a


def make_desc(gid, N, lo, hi, lengths, values=None, S=1, T=1, seed=0,
              precision=ZMC_FP32_KAHAN, mem=ZMC_MEM_HOST, first_index=0, count=-1,
              stream=None, tiles=(0, 0, 0), flags=0, keep=None, chunk_points=0):
    """Fill a zmc_scan_desc.  For ZMC_MEM_DEVICE, ``values`` is a device
    pointer (int) or a torch CUDA float64 tensor."""
    keep = keep if keep is not None else _Keep()
    d = zmc_scan_desc_init()
    lo_a = keep.arr(lo, np.float64)
    hi_a = keep.arr(hi, np.float64)
    L = keep.arr(lengths, np.int64)
    d.integrand_id, d.N, d.M = int(gid), int(N), len(L)
    d.lo, d.hi = lo_a.ctypes.data_as(_dp), hi_a.ctypes.data_as(_dp)
    d.list_len = L.ctypes.data_as(_i64p)
    if mem == ZMC_MEM_HOST:
        v = keep.arr(values, np.float64)
        d.list_vals = v.ctypes.data_as(_dp)
    else:
        ptr = values if isinstance(values, int) else values.data_ptr()
        keep.items.append(values)
        d.list_vals = ctypes.cast(ctypes.c_void_p(ptr), _dp)
    d.samples_per_point, d.trials, d.seed = int(S), int(T), int(seed) & (2 ** 64 - 1)
    d.precision, d.mem = int(precision), int(mem)
    d.first_index, d.count = int(first_index), int(count)
    d.stream = stream
    d.tile_lanes, d.tile_splits, d.tile_block = (int(x) for x in tiles)
    d.flags = int(flags)
    d.chunk_points = int(chunk_points)
    return d, keep


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(_dp)
    return ctypes.cast(ctypes.c_void_p(x.data_ptr()), _dp)


def scan(gid, N, lo, hi, lengths, values, S, T, seed, precision=ZMC_FP32_KAHAN,
         first_index=0, count=-1, tiles=(0, 0, 0), flags=0, want_sums=False,
         want_errw=True, chunk_points=0):
    """Host-memory scan through zmc_scan_ex; returns a dict of numpy arrays
    (mean, err, errw, [s1, s2]) and the zmc_scan_out."""
    d, keep = make_desc(gid, N, lo, hi, lengths, values, S, T, seed, precision,
                        ZMC_MEM_HOST, first_index, count, None, tiles, flags,
                        chunk_points=chunk_points)
    P = int(np.prod(np.asarray(lengths, np.int64)))
    n = (P - first_index) if count < 0 else count
    res = {"mean": np.empty(n), "err": np.empty(n)}
    if want_errw:
        res["errw"] = np.empty(n)
    if want_sums:
        res["s1"] = np.empty((n, T))
        res["s2"] = np.empty((n, T))
    o = zmc_scan_out()
    o.mean, o.err = _ptr(res["mean"]), _ptr(res["err"])
    o.errw = _ptr(res.get("errw"))
    o.s1, o.s2 = _ptr(res.get("s1")), _ptr(res.get("s2"))
    zmc_scan_ex(d, o)
    return res, o


def scan_device(gid, N, lo, hi, lengths, values_dev, S, T, seed, out_mean, out_err,
                out_errw=None, out_s1=None, out_s2=None, precision=ZMC_FP32_KAHAN,
                first_index=0, count=-1, stream=None, workspace=None, tiles=(0, 0, 0),
                flags=0, chunk_points=0):
    """Device-memory scan: values and outputs are torch CUDA float64 tensors;
    work is enqueued on ``stream`` (a cudaStream_t as int, or None)."""
    d, keep = make_desc(gid, N, lo, hi, lengths, values_dev, S, T, seed, precision,
                        ZMC_MEM_DEVICE, first_index, count, stream, tiles, flags,
                        chunk_points=chunk_points)
    if workspace is not None:
        d.workspace = ctypes.c_void_p(workspace.data_ptr())
        d.workspace_bytes = workspace.numel() * workspace.element_size()
    o = zmc_scan_out()
    o.mean, o.err = _ptr(out_mean), _ptr(out_err)
    o.errw, o.s1, o.s2 = _ptr(out_errw), _ptr(out_s1), _ptr(out_s2)
    zmc_scan_ex(d, o)
    return o
