"""Closed forms of f(x) = \\int_box g(y; x) dy and of \\int_box g^2 dy.

These pin the oracle from outside: each is derived by hand from the
integrand's definition (a product over dimensions, or the real/imaginary part
of a product of 1-D complex integrals), evaluated with numpy/scipy, and shares
nothing with the oracle's sampling loop.  The sine-sum case is the test
integrand of Eq. 2 and Eq. 4; on [0, a]^N it reduces to
(2 sin(a/2))^N sin(sum x + N a / 2).
"""
from __future__ import annotations

import functools

import numpy as np
from scipy.special import erf

SIGMA = 0.3
OSC_Q = 0.1

G_CONST, G_COSPROD, G_GAUSS03, G_POLY, G_OSC01, G_SINSUM = range(6)


@functools.lru_cache(maxsize=8)
def _gl(n=400):
    return np.polynomial.legendre.leggauss(n)


def _int_exp_i(a, b, lin, quad, n=400):
    """\\int_a^b exp(i (lin*y + quad*y^2)) dy by Gauss-Legendre (smooth)."""
    t, w = _gl(n)
    y = 0.5 * (b - a) * t + 0.5 * (b + a)
    return 0.5 * (b - a) * np.sum(w * np.exp(1j * (lin * y + quad * y * y)))


def _cos_int(x, a, b):
    if x == 0.0:
        return b - a
    return (np.sin(x * b) - np.sin(x * a)) / x


def _cos2_int(x, a, b):
    if x == 0.0:
        return b - a
    return 0.5 * (b - a) + (np.sin(2 * x * b) - np.sin(2 * x * a)) / (4 * x)


def _gauss_int(x, a, b, s):
    c = s * np.sqrt(2.0)
    return s * np.sqrt(np.pi / 2.0) * (erf((b - x) / c) - erf((a - x) / c))


def integral(gid, x, lo, hi):
    """\\int_box g(y; x) dy."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    x = np.asarray(x, float)
    N = lo.size
    if gid == G_CONST:
        return float(np.prod(hi - lo))
    if gid == G_COSPROD:
        return float(np.prod([_cos_int(x[k], lo[k], hi[k]) for k in range(N)]))
    if gid == G_GAUSS03:
        return float(np.prod([_gauss_int(x[k], lo[k], hi[k], SIGMA)
                              for k in range(N)]))
    if gid == G_POLY:
        return float(np.prod([(hi[k] - lo[k]) + x[k] * (hi[k] ** 3 - lo[k] ** 3) / 3
                              for k in range(N)]))
    if gid == G_OSC01:
        J = np.prod([_int_exp_i(lo[k], hi[k], x[k], OSC_Q) for k in range(N)])
        return float(J.real)
    if gid == G_SINSUM:
        J = np.prod([(np.exp(1j * hi[k]) - np.exp(1j * lo[k])) / 1j
                     for k in range(N)])
        return float((np.exp(1j * np.sum(x)) * J).imag)
    raise ValueError(gid)


def integral_sq(gid, x, lo, hi):
    """\\int_box g(y; x)^2 dy."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    x = np.asarray(x, float)
    N = lo.size
    V = float(np.prod(hi - lo))
    if gid == G_CONST:
        return V
    if gid == G_COSPROD:
        return float(np.prod([_cos2_int(x[k], lo[k], hi[k]) for k in range(N)]))
    if gid == G_GAUSS03:
        return float(np.prod([_gauss_int(x[k], lo[k], hi[k], SIGMA / np.sqrt(2.0))
                              for k in range(N)]))
    if gid == G_POLY:
        return float(np.prod([(hi[k] - lo[k])
                              + 2 * x[k] * (hi[k] ** 3 - lo[k] ** 3) / 3
                              + x[k] ** 2 * (hi[k] ** 5 - lo[k] ** 5) / 5
                              for k in range(N)]))
    if gid == G_OSC01:
        J2 = np.prod([_int_exp_i(lo[k], hi[k], 2 * x[k], 2 * OSC_Q)
                      for k in range(N)])
        return 0.5 * V + 0.5 * float(J2.real)
    if gid == G_SINSUM:
        J2 = np.prod([(np.exp(2j * hi[k]) - np.exp(2j * lo[k])) / 2j
                      for k in range(N)])
        return 0.5 * V - 0.5 * float((np.exp(2j * np.sum(x)) * J2).real)
    raise ValueError(gid)


def sigma_I(gid, x, lo, hi, S):
    """Standard deviation of one trial's estimate V * mean(g) over S samples."""
    V = float(np.prod(np.asarray(hi, float) - np.asarray(lo, float)))
    m1 = integral(gid, x, lo, hi) / V
    m2 = integral_sq(gid, x, lo, hi) / V
    var = max(m2 - m1 * m1, 0.0)
    return V * np.sqrt(var / S)


def sinsum_cube(x_sum, N, a):
    """The closed form quoted for Eq. 2 / Eq. 4 on [0, a]^N."""
    return (2 * np.sin(a / 2)) ** N * np.sin(x_sum + N * a / 2)


def tensor_gauss_legendre(gid, x, lo, hi, n=64, g=None):
    """Brute-force tensor-product quadrature of g over a small box (N <= 3)."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    N = lo.size
    t, w = _gl(n)
    nodes = [0.5 * (hi[k] - lo[k]) * t + 0.5 * (hi[k] + lo[k]) for k in range(N)]
    wts = [0.5 * (hi[k] - lo[k]) * w for k in range(N)]
    grids = np.meshgrid(*nodes, indexing="ij")
    W = np.ones_like(grids[0])
    for k, wk in enumerate(np.meshgrid(*wts, indexing="ij")):
        W = W * wk
    Y = np.stack([gk.ravel() for gk in grids], axis=1)
    vals = np.array([g(Y[i], x) for i in range(Y.shape[0])])
    return float(np.sum(W.ravel() * vals))
