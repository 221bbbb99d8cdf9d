"""User integrands (NVRTC) through the full scan path on the GPU."""
import numpy as np
import pytest

import parity
import user_sources as us
from oracle import oracle
from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc
    zmc.load()
    return zmc


def test_user_cosprod_matches_the_oracle(z):
    gid = z.zmc_integrand_register("cosprod_user", us.COSPROD, 1, 8)
    for spec in [wl.scan_cosprod_100(samples=1 << 12, trials=3),
                 wl.ScanSpec("c3", 1, 3, np.zeros(3), np.array([1.0, 1.5, 2.0]),
                             [np.linspace(0.5, 5, 4), np.linspace(1, 3, 3), np.array([2.5])],
                             1001, 3, 11)]:
        ref = oracle.default().scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                    spec.values, spec.samples, spec.trials, spec.seed,
                                    want_sums=True)
        V = float(np.prod(np.asarray(spec.hi) - np.asarray(spec.lo)))
        for prec in (2, 1, 0):
            got, o = z.scan(gid, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                            spec.samples, spec.trials, spec.seed, precision=prec)
            parity.check(got, ref, V, spec.samples, prec, "user cosprod N=%d" % spec.N)
            # the run-time-compiled kernel through a chunked scan: the same bits
            chunked, oc = z.scan(gid, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                                 spec.samples, spec.trials, spec.seed, precision=prec,
                                 chunk_points=7)
            assert oc.chunks == -(-spec.P // 7) and oc.chunks > 1
            for k in got:
                assert np.array_equal(chunked[k], got[k]), (spec.N, prec, k)


def test_new_integrand_against_its_closed_form(z):
    gid = z.zmc_integrand_register("sumx_prody", us.SUMX_PRODY, 1, 4)
    for N, M in [(2, 1), (3, 2), (4, 3)]:
        hi = np.linspace(1.0, 2.0, N)
        lists = [np.linspace(0.5, 3.0, 5)] + [np.array([0.25 * l]) for l in range(1, M)]
        lengths = [len(v) for v in lists]
        vals = np.concatenate(lists)
        got, o = z.scan(gid, N, np.zeros(N), hi, lengths, vals, 1 << 14, 4, 5)
        xs = lists[0] + sum(v[0] for v in lists[1:])
        exact = xs * np.prod(hi ** 2 / 2.0)
        assert np.all(np.abs(got["mean"] - exact) < 5 * got["errw"] + 1e-6 * np.abs(exact)), \
            (N, M, got["mean"], exact)
