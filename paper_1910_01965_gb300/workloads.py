"""Seeded synthetic inputs for parameter-grid scans.

This module only builds inputs: box bounds, parameter value lists, sample and
trial counts, seeds and request arrival times.  It holds none of the method's
arithmetic (no sampling, no integrand, no estimator), so both the CUDA path
and the CPU oracle can be fed from it without sharing any computation.

The workloads:
  scan_cosprod_100      cos(x1 y1) cos(x2 y2) on [0,1]^2, lists linspace(0.5,5,10)
                        x2, S = 2^16, T = 5, seed 0 (FP64 parity case)
  scan_gauss_1e6        exp(-sum (y-x)^2 / (2 0.3^2)) on [-1,1]^4, x1..x3 each 100
                        values from default_rng(0).uniform(-1,1) (drawn x1, x2, x3
                        in order), x4 = 0 as a list of length 1; S = 2^14, T = 4
  scan_osc_1e4          cos(sum x y + 0.1 sum y^2) on [0,2]^6, x1..x4 each
                        linspace(0.5,5,10), x5 = x6 = 1; S = 2^20, T = 8
  batch_uneven_256      256 scans, N ~ U{1..8}, P log-uniform [10, 1e5],
                        S log-uniform [2^10, 2^18] rounded to a multiple of 4,
                        integrand uniform over {cos-product, Gaussian,
                        polynomial}, T = 4, seed of scan i = i; default_rng(0)
  serving_poisson       arrivals at 500 req/s (exponential gaps, default_rng(1))
                        over a window; 99% drawn like batch_uneven_256, 1% large
                        (N = 3, L = (465, 465, 463), S = 2^12, T = 4)
  sinsum_table1         the sine-sum test of Eq. 2 (Sec. 3.1): lists {0..99},
                        box [0,10]^N, S = 10^4
  sinsum_table2         the sine-sum test of Eq. 4 (Sec. 3.2): M = 4, N = 6,
                        lists {0..99}, box [0,1]^6, S = 10^5
  registry_scan         one scan per (integrand, N) of the registry, ~10^5
                        points x 4 trials x 2^15 samples (per-kernel sweeps)
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

G_CONST, G_COSPROD, G_GAUSS03, G_POLY, G_OSC01, G_SINSUM = range(6)


@dataclasses.dataclass
class ScanSpec:
    """One scan request: integrand, box, parameter lists, S, T, seed."""
    name: str
    integrand_id: int
    N: int
    lo: np.ndarray            # [N] float64
    hi: np.ndarray            # [N] float64
    lists: List[np.ndarray]   # M arrays of float64
    samples: int              # S
    trials: int               # T
    seed: int

    @property
    def M(self) -> int:
        return len(self.lists)

    @property
    def lengths(self) -> np.ndarray:
        return np.array([len(v) for v in self.lists], dtype=np.int64)

    @property
    def values(self) -> np.ndarray:
        return np.concatenate([np.asarray(v, np.float64) for v in self.lists])

    @property
    def P(self) -> int:
        return int(np.prod(self.lengths))

    @property
    def evals(self) -> int:
        """Integrand evaluations of the whole scan: P * T * S."""
        return self.P * self.trials * self.samples

    def describe(self) -> dict:
        return {"workload": self.name, "integrand": self.integrand_id, "N": self.N,
                "M": self.M, "lengths": [int(v) for v in self.lengths],
                "grid_points": self.P, "samples": self.samples,
                "trials": self.trials, "seed": self.seed}


def scan_cosprod_100(samples: int = 1 << 16, trials: int = 5) -> ScanSpec:
    x = np.linspace(0.5, 5.0, 10)
    return ScanSpec("cosprod_N2_P100_S2^16_T5", G_COSPROD, 2, np.zeros(2),
                    np.ones(2), [x.copy(), x.copy()], samples, trials, 0)


def scan_gauss_1e6(samples: int = 1 << 14, trials: int = 4) -> ScanSpec:
    rng = np.random.default_rng(0)
    x1 = rng.uniform(-1.0, 1.0, 100)
    x2 = rng.uniform(-1.0, 1.0, 100)
    x3 = rng.uniform(-1.0, 1.0, 100)
    return ScanSpec("gauss03_N4_P1e6_S2^14_T4", G_GAUSS03, 4, -np.ones(4),
                    np.ones(4), [x1, x2, x3, np.zeros(1)], samples, trials, 0)


def scan_osc_1e4(samples: int = 1 << 20, trials: int = 8) -> ScanSpec:
    x = np.linspace(0.5, 5.0, 10)
    lists = [x.copy() for _ in range(4)] + [np.ones(1), np.ones(1)]
    return ScanSpec("osc01_N6_P1e4_S2^20_T8", G_OSC01, 6, np.zeros(6),
                    2.0 * np.ones(6), lists, samples, trials, 0)


def _uneven_scan(rng: np.random.Generator, index: int, trials: int = 4) -> ScanSpec:
    N = int(rng.integers(1, 9))
    P_target = math.exp(rng.uniform(math.log(10.0), math.log(1e5)))
    S = math.exp(rng.uniform(math.log(2.0 ** 10), math.log(2.0 ** 18)))
    S = max(4, int(round(S / 4.0)) * 4)
    gid = [G_COSPROD, G_GAUSS03, G_POLY][int(rng.integers(0, 3))]
    m = min(N, 3)
    side = max(1, int(round(P_target ** (1.0 / m))))
    lens = [side] * m + [1] * (N - m)
    if gid == G_GAUSS03:
        lo, hi = -np.ones(N), np.ones(N)
        lists = [rng.uniform(-1.0, 1.0, L) for L in lens]
    else:
        lo, hi = np.zeros(N), np.ones(N)
        lists = [rng.uniform(0.5, 5.0, L) for L in lens]
    return ScanSpec("uneven_%03d" % index, gid, N, lo, hi, lists, S, trials, index)


def batch_uneven_256(count: int = 256, trials: int = 4, seed: int = 0) -> List[ScanSpec]:
    rng = np.random.default_rng(seed)
    return [_uneven_scan(rng, i, trials) for i in range(count)]


def large_scan(index: int, samples: int = 1 << 12, trials: int = 4,
               lengths=(465, 465, 463)) -> ScanSpec:
    rng = np.random.default_rng(10_000 + index)
    lists = [rng.uniform(0.5, 5.0, L) for L in lengths]
    return ScanSpec("large_%03d" % index, G_COSPROD, 3, np.zeros(3), np.ones(3),
                    lists, samples, trials, 1_000_000 + index)


@dataclasses.dataclass
class Arrival:
    t: float          # seconds after the start of the window
    spec: ScanSpec
    large: bool


def serving_poisson(rate: float = 500.0, window_s: float = 10.0,
                    large_fraction: float = 0.01, seed: int = 1,
                    large_lengths=(465, 465, 463),
                    max_requests: Optional[int] = None) -> List[Arrival]:
    rng = np.random.default_rng(seed)
    out: List[Arrival] = []
    t = 0.0
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= window_s or (max_requests is not None and i >= max_requests):
            break
        if rng.uniform() < large_fraction:
            out.append(Arrival(t, large_scan(i, lengths=large_lengths), True))
        else:
            out.append(Arrival(t, _uneven_scan(rng, i), False))
        i += 1
    return out


def sinsum_table1(M: int, N: int, samples: int = 10_000, trials: int = 1,
                  seed: int = 0) -> ScanSpec:
    lists = [np.arange(100.0) for _ in range(M)]
    return ScanSpec("sinsum_table1_M%d_N%d" % (M, N), G_SINSUM, N, np.zeros(N),
                    10.0 * np.ones(N), lists, samples, trials, seed)


def sinsum_table2(samples: int = 100_000, trials: int = 1, seed: int = 0) -> ScanSpec:
    lists = [np.arange(100.0) for _ in range(4)]
    return ScanSpec("sinsum_table2_M4_N6", G_SINSUM, 6, np.zeros(6), np.ones(6),
                    lists, samples, trials, seed)


def registry_scan(gid: int, N: int, points: int = 100_000, samples: int = 1 << 15,
                  trials: int = 4) -> ScanSpec:
    """One scan of integrand `gid` at dimension N for per-kernel throughput
    sweeps: M = N lists, the first min(N, 3) of length round(points^(1/min(N,3)))
    and the rest of length 1, drawn from default_rng(100 + 10 gid + N).  Boxes
    and parameter ranges as in the workloads above: cos-product and polynomial
    on [0,1]^N with x ~ U[0.5, 5]; Gaussian on [-1,1]^N with x ~ U[-1, 1];
    oscillatory on [0,2]^N with x ~ U[0.5, 5]; sine-sum on [0,1]^N with
    integer x in {0..99}."""
    rng = np.random.default_rng(100 + 10 * gid + N)
    m = min(N, 3)
    side = max(1, int(round(points ** (1.0 / m))))
    lens = [side] * m + [1] * (N - m)
    if gid == G_GAUSS03:
        lo, hi = -np.ones(N), np.ones(N)
        lists = [rng.uniform(-1.0, 1.0, L) for L in lens]
    elif gid == G_OSC01:
        lo, hi = np.zeros(N), 2.0 * np.ones(N)
        lists = [rng.uniform(0.5, 5.0, L) for L in lens]
    elif gid == G_SINSUM:
        lo, hi = np.zeros(N), np.ones(N)
        lists = [rng.integers(0, 100, L).astype(np.float64) for L in lens]
    else:
        lo, hi = np.zeros(N), np.ones(N)
        lists = [rng.uniform(0.5, 5.0, L) for L in lens]
    names = {G_CONST: "const", G_COSPROD: "cosprod", G_GAUSS03: "gauss03", G_POLY: "poly",
             G_OSC01: "osc01", G_SINSUM: "sinsum"}
    P = int(np.prod(lens))
    return ScanSpec("%s_N%d_P%d_S%d_T%d" % (names[gid], N, P, samples, trials), gid, N, lo, hi,
                    lists, samples, trials, 0)


def sample_points(P: int, count: int, seed: int = 12345) -> np.ndarray:
    """Sorted, distinct, seeded flat indices in [0, P), including 0 and P-1."""
    count = min(count, P)
    rng = np.random.default_rng(seed)
    pts = set(int(v) for v in rng.choice(P, size=count, replace=False))
    pts.discard(0)
    pts.discard(P - 1)
    pts = sorted(pts)[: max(0, count - 2)] + [0, P - 1]
    return np.array(sorted(set(pts)), dtype=np.int64)
