"""Tolerances for comparing the CUDA path with the FP64 oracle.

Scale of a point: R = V * sqrt(mean_t s2_t / S), the root-mean-square of g
times the volume, from the oracle's own sums; comparisons use
max(|oracle mean|, R) so that points where f(x) is near zero (the cosine and
sine integrands) are judged against the size of what was summed.

  FP64 path:  |mean - oracle| <= 1e-12 * max(|oracle|, R),
              |err  - oracle| <= 1e-12 * max(err, R)
  FP32 path:  |mean - oracle| <= 1e-5 * max(|oracle|, R)  and
              |mean - oracle| <= 0.05 standard errors,
              |err  - oracle| <= 0.05 standard errors
The standard error here is the oracle's errw, pooled over all T*S samples:
the spread over T trials (err) estimates the same quantity but from T values
only, so with T = 2 or 3 it can be arbitrarily small by chance.
"""
import numpy as np


def scale(ref, V, S):
    R = V * np.sqrt(np.mean(ref["s2"], axis=1) / S)
    return np.maximum(np.abs(ref["mean"]), R), R


def check(got, ref, V, S, precision, what=""):
    """Raise AssertionError with the worst offender if out of tolerance.
    Returns a dict of the worst scaled deviations (for reports)."""
    sc, R = scale(ref, V, S)
    dm = np.abs(got["mean"] - ref["mean"])
    report = {"max_dmean_scaled": float(np.max(dm / sc)) if dm.size else 0.0}
    if precision == 0:  # FP64
        bad = dm > 1e-12 * sc
        assert not np.any(bad), "%s FP64 mean: worst %.3g (scaled) at %d" % (
            what, np.max(dm / sc), int(np.argmax(dm / sc)))
        if np.all(np.isfinite(ref["err"])):
            de = np.abs(got["err"] - ref["err"])
            lim = 1e-12 * np.maximum(ref["err"], R)
            assert np.all(de <= lim), "%s FP64 err: worst %.3g" % (what, np.max(de / lim))
    else:
        bad = dm > 1e-5 * sc
        assert not np.any(bad), "%s FP32 mean: worst %.3g of scale at %d" % (
            what, np.max(dm / sc), int(np.argmax(dm / sc)))
        se = ref["errw"]
        ok = np.isfinite(se) & (se > 0)
        if np.any(ok):
            zs = dm[ok] / se[ok]
            report["max_dmean_in_stderr"] = float(np.max(zs))
            assert np.all(zs <= 0.05), "%s FP32 mean: %.3g standard errors at %d" % (
                what, np.max(zs), int(np.flatnonzero(ok)[np.argmax(zs)]))
            if np.all(np.isfinite(ref["err"][ok])):
                de = np.abs(got["err"][ok] - ref["err"][ok]) / se[ok]
                report["max_derr_in_stderr"] = float(np.max(de))
                assert np.all(de <= 0.05), "%s FP32 err: %.3g standard errors" % (
                    what, np.max(de))
    if "errw" in got and "errw" in ref and np.all(np.isfinite(ref["errw"])):
        tol = 1e-12 if precision == 0 else 1e-3
        dw = np.abs(got["errw"] - ref["errw"]) / np.maximum(ref["errw"], 1e-300)
        ok = (dw <= tol) | (np.abs(got["errw"] - ref["errw"]) <= tol * R / np.sqrt(S))
        assert np.all(ok), "%s errw: worst relative %.3g" % (what, np.max(dw))
    return report
