"""The single-scan tile planner's choices on this device (ZMC_F_PLAN_ONLY).

Lanes per unit-split: the largest power of two <= 32 leaving each lane >= 512
sample groups (64 for plain FP32 lane sums), doubled while the launch is
short of 16 waves of resident threads and each lane keeps >= 64 groups; then
splits up to 16 waves, never below 64 groups per lane.  The rule is restated
here from the device's SM count and threads per SM and compared with the
library's plan; no autotuner entry is recorded in this process.
"""
import numpy as np
import pytest

from paper_1910_01965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zmc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01965_gb300 import zmc as z
    z.load()
    z.zmc_autotune_reset()
    return z


def _rule(N, S, T, count, sm, tps, prec):
    G = 1 if N % 5 == 0 else 5
    Q = (S + G - 1) // G
    units = max(1, count * T)
    want = 16 * max(1, sm) * max(256, tps)
    min_groups = 64 if prec == 1 else 512
    lanes = 32
    while lanes > 1 and Q // lanes < min_groups:
        lanes >>= 1
    while lanes < 32 and units * lanes < want and Q // (2 * lanes) >= 64:
        lanes <<= 1
    splits = -(-want // (units * lanes))
    splits = max(1, min(splits, max(1, Q // (lanes * 64))))
    splits = min(splits, max(1, Q))
    return lanes, splits, 256


def test_planner_matches_its_rule(zmc):
    info = zmc.zmc_device_info_get()
    head = wl.scan_gauss_1e6()
    cases = [(head, 2), (head, 1), (head, 0)]
    r = np.random.default_rng(3)
    for P, S, N in [(1000, 1 << 14, 4), (10, 1 << 18, 2), (50_000, 1 << 11, 3), (200, 777, 5),
                    (3, 1 << 20, 8), (10 ** 5, 1 << 15, 6)]:
        m = min(N, 3)
        side = max(1, int(round(P ** (1.0 / m))))
        lists = [r.uniform(0.5, 5, side) for _ in range(m)] + [np.ones(1)] * (N - m)
        spec = wl.ScanSpec("plan", wl.G_COSPROD, N, np.zeros(N), np.ones(N), lists, S, 4, 1)
        cases += [(spec, 2), (spec, 1)]
    for spec, prec in cases:
        res, o = zmc.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                          spec.values, spec.samples, spec.trials, spec.seed, precision=prec,
                          flags=zmc.ZMC_F_PLAN_ONLY)
        want = _rule(spec.N, spec.samples, spec.trials, spec.P, info.sm_count,
                     info.max_threads_per_sm, prec)
        assert (o.tile_lanes, o.tile_splits, o.tile_block) == want, (spec.P, spec.samples,
                                                                    spec.N, prec)
        assert o.launches == 0
    # the headline grid: four long lanes in the compensated path, 32 in plain FP32
    res, o = zmc.scan(head.integrand_id, head.N, head.lo, head.hi, head.lengths, head.values,
                      head.samples, head.trials, head.seed, precision=2,
                      flags=zmc.ZMC_F_PLAN_ONLY)
    assert o.tile_lanes == 4 and o.tile_splits == 1
