"""The CUDA path against the values printed in Table 1 (Sec. 3.1).

delta r (Eq. 3, |f| in the denominator) of the sine-sum test of Eq. 2 on
[0,10]^N with lists {0..99}^M.  The printed values are matched by 10^5
samples per point (see the oracle's golden test for the reading): with 10^4
grid points and more, delta r is stable to a few per cent.
"""
import os

import numpy as np
import pytest

from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _table1():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table1_delta_r.txt")):
        if line.strip() and not line.startswith("#"):
            M, N, d = line.split()
            rows[(int(M), int(N))] = float(d)
    return rows


@pytest.mark.parametrize("M", [2, 3])
def test_delta_r_matches_table1(M):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc
    table = _table1()
    v = np.arange(100.0)
    xs = np.zeros(1)
    for _ in range(M):
        xs = (xs[:, None] + v[None, :]).ravel()
    for N in (1, 2, 3, 4):
        spec = wl.sinsum_table1(M, N, samples=100_000)
        mean, err = zmc.zmc_scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                 spec.values, spec.samples, spec.trials, spec.seed)
        fth = (2 * np.sin(5.0)) ** N * np.sin(xs + N * 5.0)
        dr = np.mean(np.abs(fth - mean) / np.abs(fth))
        assert 0.92 < dr / table[(M, N)] < 1.08, (M, N, dr, table[(M, N)])
