"""Pins of the FP64 oracle against things other than itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` (a loaded build) and raises
AssertionError when the build disagrees with an outside fact:
  - Philox4x32-10, the counter layout and the cut of each call's 128 output
    bits into five 23-bit fields: Triton's own Philox (a third-party
    implementation, run in its CPU interpreter) and Python integers;
  - the uniform map and the map into the box: exact rational arithmetic;
  - grid decode (Sec. 2, C order): numpy's unravel_index / meshgrid('ij');
  - the estimator: closed forms of f(x) and of the variance of g (the sine-sum
    case is the test integrand of Eq. 2 / Eq. 4), the constant integrand's
    exact volume, error calibration, 1/sqrt(S) scaling, tensor Gauss-Legendre
    quadrature on tiny grids, and a brute-force recomputation on tiny inputs
    from Triton's Philox words.
The same functions run against deliberately broken copies of the oracle in
test_oracle_mutants.py, to show that each plausible mistake fails a pin.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np

import closed_forms as cf

MASK32 = 0xFFFFFFFF
HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# Reference Philox words from Triton (computed once per session).
# ---------------------------------------------------------------------------
def philox_requests():
    """Counters/keys the Philox pins use (seeded, with edge values)."""
    rng = np.random.default_rng(20191004)
    ctr = [[0, 0, 0, 0], [1, 0, 0, 0], [MASK32] * 4, [0, 1, 0, 0],
           [0, 0, 1, 0], [0, 0, 0, 1]]
    seed = [0, 0, 2 ** 64 - 1, 0, 0, 0]
    for _ in range(58):
        ctr.append([int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)])
        seed.append(int(rng.integers(0, 2 ** 63, dtype=np.int64)) * 2
                    + int(rng.integers(0, 2)))
    # Counter layout cases: (seed, p, t, w) -> ctr (w>>2, t, p lo, p hi).
    layout = [(0, 0, 0, 0), (0, 0, 0, 5), (7, 3, 2, 11), (2 ** 40 + 12345, 1, 0, 7),
              (123, 2 ** 33 + 5, 3, 2 ** 33 + 9), (2 ** 64 - 2, 2 ** 61, 2 ** 31 - 1, 3)]
    for _ in range(26):
        layout.append((int(rng.integers(0, 2 ** 63)), int(rng.integers(0, 2 ** 62)),
                       int(rng.integers(0, 2 ** 31)), int(rng.integers(0, 2 ** 34))))
    for (s, p, t, w) in layout:
        ctr.append([w >> 2, t, p & MASK32, p >> 32])
        seed.append(s)
        # the same index read as a field index, and the fields of a 3-D sample
        for i in [w] + [(w // 3) * 3 + k for k in range(3)]:
            ctr.append([i // 5, t, p & MASK32, p >> 32])
            seed.append(s)
    for j in range(3):  # all slots of three consecutive calls
        ctr.append([j, 2, 3, 0])
        seed.append(7)
    return ctr, seed, layout


def brute_cases():
    """Tiny brute-force cases: (gid, N, lo, hi, lengths, values, S, T, seed, points)."""
    big = 70000  # 70000^2 > 2^32, exercises the high counter word of p
    return [
        (cf.G_COSPROD, 2, [0.0, -0.5], [1.0, 1.5], [2, 1], [0.7, 2.5, -1.25], 5, 3,
         2 ** 40 + 12345, [0, 1]),
        (cf.G_SINSUM, 3, [0.0, 1.0, -2.0], [10.0, 3.0, 0.5], [3], [0.0, 1.0, 2.0], 7, 2,
         99, [0, 2]),
        (cf.G_GAUSS03, 2, [-1.0, -0.5], [1.0, 1.0], [big, big],
         list(np.linspace(-1, 1, big)) * 2, 4, 2, 5, [big * big - 1, 2 ** 32 + 17]),
    ]


def triton_words(ctr, seed):
    """Run Triton's Philox (CPU interpreter) in a child process."""
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "philox_triton_ref.py")],
                          input=json.dumps({"ctr": ctr, "seed": seed}),
                          capture_output=True, text=True, env=env, timeout=600)
    if proc.returncode != 0:
        raise RuntimeError("triton reference failed: " + proc.stderr[-2000:])
    return json.loads(proc.stdout)


def reference_tables():
    """All reference words the pins need, from one Triton run."""
    ctr, seed, layout = philox_requests()
    # brute-force cases need every word they use
    brute_keys = []
    for (gid, N, lo, hi, L, vals, S, T, sd, pts) in brute_cases():
        for p in pts:
            for t in range(T):
                for j in range((S * N + 4) // 5):
                    brute_keys.append((sd, p, t, j))
    for (sd, p, t, j) in brute_keys:
        ctr.append([j, t, p & MASK32, p >> 32])
        seed.append(sd)
    out = triton_words(ctr, seed)
    table = {}
    for c, s, o in zip(ctr, seed, out):
        table[(tuple(c), s)] = o
    return {"table": table, "layout": layout, "ctr": ctr, "seed": seed}


def _ref_word(ref, seed, p, t, w):
    return ref["table"][((w >> 2, t, p & MASK32, p >> 32), seed)][w & 3]


def _ref_field(ref, seed, p, t, i):
    """Field i: bits 23m..23m+22 (m = i mod 5) of call i // 5's four words
    read as one 128-bit integer, lowest word first."""
    r = ref["table"][((i // 5, t, p & MASK32, p >> 32), seed)]
    block = r[0] | (r[1] << 32) | (r[2] << 64) | (r[3] << 96)
    return (block >> (23 * (i % 5))) & (2 ** 23 - 1)


# ---------------------------------------------------------------------------
# RNG pins
# ---------------------------------------------------------------------------
def pin_philox(O, ref):
    n = 0
    for (c, s), o in ref["table"].items():
        got = O.philox4x32_10(c, [s & MASK32, s >> 32])
        assert got == o, "philox mismatch ctr=%s seed=%d: %s vs %s" % (c, s, got, o)
        n += 1
    assert n > 60


def pin_word_layout(O, ref):
    for (s, p, t, w) in ref["layout"]:
        assert O.word(s, p, t, w) == _ref_word(ref, s, p, t, w), (s, p, t, w)


def pin_field_layout(O, ref):
    for (s, p, t, w) in ref["layout"]:
        assert O.field(s, p, t, w) == _ref_field(ref, s, p, t, w), (s, p, t, w)
    # every slot of one call, and the two calls around a call boundary
    s, p, t = 7, 3, 2
    seen = set()
    for i in range(15):
        v = O.field(s, p, t, i)
        assert 0 <= v < 2 ** 23
        seen.add(v)
        assert v == _ref_field(ref, s, p, t, i), i
    assert len(seen) == 15


def pin_uniform(O):
    rng = np.random.default_rng(1)
    vs = [0, 1, 2, 2 ** 22 - 1, 2 ** 22, 2 ** 23 - 2, 2 ** 23 - 1] + \
        [int(v) for v in rng.integers(0, 2 ** 23, 200)]
    for v in vs:
        u = O.uniform(v)
        exact = Fraction(2 * v + 1, 2 ** 24)
        assert Fraction(u) == exact, (v, u)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exactly representable in FP32


def pin_sample_y(O, ref):
    # y_k = lo_k + (hi_k - lo_k) * u, rounded once (the box map of direct MC),
    # u from field s*N + k
    lo = [0.0, -0.5, -3.0]
    hi = [1.0, 1.5, 7.25]
    for (s, p, t, w) in ref["layout"][:12]:
        N = 3
        samp = w // N
        y = O.sample_y(N, lo, hi, s, p, t, samp)
        for k in range(N):
            v = _ref_field(ref, s, p, t, samp * N + k)
            u = Fraction(2 * v + 1, 2 ** 24)
            wdt = Fraction(hi[k] - lo[k])  # the width as a double
            want = float(Fraction(lo[k]) + wdt * u)
            assert y[k] == want, (s, p, t, samp, k, y[k], want)


# ---------------------------------------------------------------------------
# Grid decode (Sec. 2): Cartesian product of the lists, C order
# ---------------------------------------------------------------------------
def pin_decode(O):
    for lengths in [(3, 1, 4, 5), (7, 11, 13), (1,), (100, 100, 100, 1), (2, 3)]:
        P = int(np.prod(lengths))
        idx = range(P) if P <= 5000 else \
            list(range(50)) + list(np.random.default_rng(3).integers(0, P, 300))
        for p in idx:
            d = O.decode(lengths, int(p))
            assert tuple(d) == tuple(int(v) for v in np.unravel_index(int(p), lengths)), \
                (lengths, p, d)
    lists = [np.array([0.5, 1.5, 2.5]), np.array([-1.0, 4.0]), np.array([9.0, 8.0, 7.0, 6.0])]
    lengths = [len(v) for v in lists]
    vals = np.concatenate(lists)
    mesh = np.meshgrid(*lists, indexing="ij")
    flat = np.stack([m.ravel() for m in mesh], axis=1)
    for p in range(flat.shape[0]):
        assert np.array_equal(O.grid_point(lengths, vals, p), flat[p])


# ---------------------------------------------------------------------------
# The estimator
# ---------------------------------------------------------------------------
def estimator_cases():
    """(gid, N, lo, hi, lists): non-cubic boxes, lists of unequal lengths."""
    r = np.random.default_rng(11)
    return [
        (cf.G_COSPROD, 2, [0.0, -0.5], [1.0, 1.5],
         [np.linspace(0.5, 5, 10), np.linspace(-2, 3, 7)]),
        (cf.G_COSPROD, 3, [0.0, -1.0, 0.2], [1.0, 0.5, 2.0],
         [np.linspace(0.5, 3, 3), np.linspace(-1, 2, 4), np.linspace(0.1, 1.5, 5)]),
        (cf.G_GAUSS03, 4, [-1.0, -1.0, -0.5, -1.0], [1.0, 0.8, 1.0, 1.2],
         [r.uniform(-1, 1, 4), r.uniform(-1, 1, 3), r.uniform(-1, 1, 5), r.uniform(-1, 1, 2)]),
        (cf.G_POLY, 3, [0.0, 0.5, -1.0], [1.0, 2.0, 1.0],
         [r.uniform(0.5, 5, 5), r.uniform(0.5, 5, 4), r.uniform(0.5, 5, 3)]),
        (cf.G_OSC01, 3, [0.0, 0.0, 0.5], [2.0, 1.5, 2.0],
         [r.uniform(0.5, 5, 4), r.uniform(0.5, 5, 5), r.uniform(0.5, 5, 3)]),
        (cf.G_SINSUM, 2, [0.0, 1.0], [10.0, 3.0],
         [np.arange(5.0), np.arange(4.0), np.array([0.5, 1.5])]),
    ]


def _run_case(O, case, S, T, seed=0):
    gid, N, lo, hi, lists = case
    lengths = [len(v) for v in lists]
    vals = np.concatenate(lists)
    res = O.scan(gid, N, lo, hi, lengths, vals, S, T, seed)
    mesh = np.meshgrid(*lists, indexing="ij")
    X = np.stack([m.ravel() for m in mesh], axis=1)
    f = np.array([cf.integral(gid, X[i], lo, hi) for i in range(X.shape[0])])
    sig = np.array([cf.sigma_I(gid, X[i], lo, hi, S) for i in range(X.shape[0])])
    return res, f, sig


def pin_const(O):
    # g = 1: the estimate is the exact volume, with zero spread.
    lo, hi = [0.0, -2.0, 1.0], [4.0, 2.0, 3.0]  # V = 4*4*2 = 32
    res = O.scan(cf.G_CONST, 3, lo, hi, [2, 3], [0.0, 1.0, 5.0, 6.0, 7.0], 1000, 4, 9)
    assert np.all(res["mean"] == 32.0), res["mean"]
    assert np.all(res["err"] == 0.0)
    assert np.all(res["errw"] == 0.0)
    res1 = O.scan(cf.G_CONST, 1, [0.25], [1.0], [1], [0.0], 3, 1, 0)
    assert res1["mean"][0] == 0.75 and np.isnan(res1["err"][0])


def pin_closed_forms(O, S=1 << 13, T=5):
    """Estimates are unbiased for the closed forms: z ~ N(0, 1)."""
    for case in estimator_cases():
        res, f, sig = _run_case(O, case, S, T)
        z = (res["mean"] - f) / (sig / np.sqrt(T))
        assert np.all(np.isfinite(z)), case[0]
        assert np.max(np.abs(z)) < 5.0, (case[0], np.max(np.abs(z)))
        assert 0.4 < np.mean(z * z) < 1.8, (case[0], np.mean(z * z))


def pin_err_calibration(O):
    """err (spread over trials) matches the theoretical sigma_I / sqrt(T)."""
    for T, lo_b, hi_b in [(2, 0.7, 1.3), (3, 0.78, 1.22), (8, 0.85, 1.15)]:
        ratios = []
        for case in estimator_cases():
            res, f, sig = _run_case(O, case, 1 << 10, T, seed=17)
            ratios.append(res["err"] ** 2 / (sig ** 2 / T))
        r = np.concatenate(ratios)
        assert lo_b < np.mean(r) < hi_b, (T, np.mean(r), r.size)


def pin_errw_calibration(O, S=1 << 13, T=5):
    """errw (pooled within-trial) matches V*sqrt(Var g/(T S)) closely."""
    for case in estimator_cases():
        res, f, sig = _run_case(O, case, S, T)
        r = res["errw"] / (sig / np.sqrt(T))
        assert abs(np.mean(r) - 1) < 0.05, (case[0], np.mean(r))
        assert np.all(np.abs(r - 1) < 0.3), (case[0], r.min(), r.max())


def pin_inv_sqrt_S(O):
    """Accuracy depends only on the number of samples (Sec. 3.2): 1/sqrt(S)."""
    case = estimator_cases()[0]
    gid, N, lo, hi, lists = case
    lengths = [len(v) for v in lists]
    vals = np.concatenate(lists)
    a = O.scan(gid, N, lo, hi, lengths, vals, 1 << 12, 2, 5)["errw"]
    b = O.scan(gid, N, lo, hi, lengths, vals, 1 << 14, 2, 5)["errw"]
    assert 0.48 < np.median(b / a) < 0.52, np.median(b / a)


def pin_quadrature(O):
    """Tiny grids: MC at large S agrees with tensor Gauss-Legendre quadrature."""
    cases = [(cf.G_POLY, 2, [0.0, -1.0], [1.0, 0.5], [[0.5, 4.0], [2.5]]),
             (cf.G_OSC01, 2, [0.0, 0.5], [2.0, 2.0], [[1.0], [0.5, 4.5]])]
    for gid, N, lo, hi, lists in cases:
        lengths = [len(v) for v in lists]
        vals = np.concatenate([np.asarray(v, float) for v in lists])
        res = O.scan(gid, N, lo, hi, lengths, vals, 1 << 20, 2, 3)
        mesh = np.meshgrid(*[np.asarray(v, float) for v in lists], indexing="ij")
        X = np.stack([m.ravel() for m in mesh], axis=1)
        for i in range(X.shape[0]):
            q = cf.tensor_gauss_legendre(gid, X[i], lo, hi, n=48,
                                         g=lambda y, x: O.integrand(gid, y, x))
            assert abs(res["mean"][i] - q) < 5 * res["errw"][i], \
                (gid, i, res["mean"][i], q, res["errw"][i])


def _numpy_g(gid, y, x):
    if gid == cf.G_COSPROD:
        return float(np.prod(np.cos(x * y)))
    if gid == cf.G_SINSUM:
        return float(np.sin(np.sum(y) + np.sum(x)))
    if gid == cf.G_GAUSS03:
        return float(np.exp(-np.sum((y - x) ** 2) / (2 * 0.3 * 0.3)))
    raise ValueError(gid)


def pin_bruteforce(O, ref):
    """Tiny inputs recomputed from Triton's Philox words and exact arithmetic."""
    for (gid, N, lo, hi, L, vals, S, T, seed, pts) in brute_cases():
        vals = np.asarray(vals, float)
        res = O.scan_points(gid, N, lo, hi, L, vals, S, T, seed, pts, want_sums=True)
        V = float(np.prod(np.asarray(hi) - np.asarray(lo)))
        for i, p in enumerate(pts):
            x = np.array([vals[int(np.sum(L[:m])) + d]
                          for m, d in enumerate(np.unravel_index(p, L))])
            I = []
            pooled = 0.0
            for t in range(T):
                g = []
                for s in range(S):
                    y = np.empty(N)
                    for k in range(N):
                        v = _ref_field(ref, seed, p, t, s * N + k)
                        u = Fraction(2 * v + 1, 2 ** 24)
                        y[k] = float(Fraction(lo[k]) + Fraction(hi[k] - lo[k]) * u)
                    g.append(_numpy_g(gid, y, x))
                g = np.array(g)
                s1, s2 = float(np.sum(g)), float(np.sum(g * g))
                assert abs(res["s1"][i, t] - s1) <= 1e-13 * max(1.0, np.sum(np.abs(g)))
                assert abs(res["s2"][i, t] - s2) <= 1e-13 * max(1.0, s2)
                I.append(V * s1 / S)
                pooled += (s2 - s1 * s1 / S) / (S - 1)
            I = np.array(I)
            mean = I.mean()
            err = np.sqrt(np.sum((I - mean) ** 2) / (T * (T - 1)))
            errw = V * np.sqrt(pooled / T / (T * S))
            scale = V * max(1.0, np.sqrt(np.mean(res["s2"][i]) / S))
            assert abs(res["mean"][i] - mean) <= 1e-12 * scale, (gid, p)
            assert abs(res["err"][i] - err) <= 1e-9 * max(err, 1e-300) + 1e-14 * scale
            assert abs(res["errw"][i] - errw) <= 1e-9 * errw + 1e-14 * scale


def pin_validation(O):
    """Argument checks of the oracle: bad inputs are refused, not computed."""
    import pytest
    for args in [
        (cf.G_COSPROD, 2, [0, 0], [1, 1], [2], [1.0, 2.0], 4, 1, 0),      # M != N
        (cf.G_CONST, 1, [1.0], [1.0], [1], [0.0], 4, 1, 0),               # empty box
        (cf.G_CONST, 1, [0.0], [1.0], [0], [], 4, 1, 0),                  # empty list
        (cf.G_CONST, 1, [0.0], [1.0], [1], [0.0], 0, 1, 0),               # S = 0
        (cf.G_CONST, 1, [0.0], [1.0], [1], [0.0], 4, 0, 0),               # T = 0
        (17, 1, [0.0], [1.0], [1], [0.0], 4, 1, 0),                       # unknown id
    ]:
        with pytest.raises(ValueError):
            O.scan_points(*args, [0])


def all_pins(O, ref, fast=False):
    """Run every pin (used by the mutant test)."""
    pin_philox(O, ref)
    pin_word_layout(O, ref)
    pin_field_layout(O, ref)
    pin_uniform(O)
    pin_sample_y(O, ref)
    pin_decode(O)
    pin_const(O)
    pin_bruteforce(O, ref)
    pin_closed_forms(O)
    pin_err_calibration(O)
    pin_errw_calibration(O)
    if not fast:
        pin_inv_sqrt_S(O)
        pin_quadrature(O)
