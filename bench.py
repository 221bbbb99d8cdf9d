#!/usr/bin/env python3
"""Benchmark of the parameter-grid direct Monte Carlo scan on GB300.

One step = one full scan of the workload (every grid point, every trial,
every sample: the sampling kernel and the finalize kernel) with inputs and
outputs resident in device memory.  Default workload: the Gaussian integrand
on [-1,1]^4 over a 100 x 100 x 100 x 1 parameter grid, 2^14 samples x 4
trials per point, FP32 evaluation with Kahan-compensated lane sums.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MC evals/s on 1 GB300 and % FP32/SFU peak vs FP64 path; "
          "p50/p99 scan latency")

# Algorithmic operations per integrand evaluation, from the method's steps
# (counted per sample of N dimensions; see the measurement section of the
# design notes): Philox4x32-10 = 10 rounds x (2 wide multiplies + 2 three-input
# XORs) = 40 per call, and a call gives five 23-bit fields -> 8 N; field -> u
# and u -> y: 2 N; the integrand; the lane accumulation of g and g^2.
INTEGRAND_OPS = {
    0: lambda N: 0,              # const (draws no samples)
    1: lambda N: 3 * N - 1,      # cos-product: x*y, cos, product
    2: lambda N: 2 * N + 2,      # Gaussian: (y-x), square-accumulate; scale, exp
    3: lambda N: 3 * N - 1,      # polynomial: y^2, 1 + x y^2, product
    4: lambda N: 2 * N + 2,      # oscillatory: x*y and y^2 accumulations; combine, cos
    5: lambda N: N + 2,          # sine-sum: y accumulation; + sum x, sin
}
ACCUM_OPS = {0: 2, 1: 2, 2: 9}   # FP64, FP32: add + fma; Kahan: g^2 + 2 x 4


def ops_per_eval(gid: int, N: int, prec: int) -> int:
    rng = 0 if gid == 0 else 8 * N + 2 * N
    return rng + INTEGRAND_OPS[gid](N) + ACCUM_OPS[prec]


# The same algorithmic operations split by the SM pipe that executes them:
# Philox's 20 wide multiplies per call on the FMA-heavy pipe (4 N per
# evaluation), its 20 three-input XORs and one logic operation per field on the
# ALU (5 N), the box map, the integrand's arithmetic and the accumulation on the
# FP32 (or FP64) pipe, and the integrand's cos/sin/exp on the XU.
INTEGRAND_FP = {1: lambda N: 2 * N - 1, 2: lambda N: 2 * N + 1, 3: lambda N: 3 * N - 1,
                4: lambda N: 2 * N + 1, 5: lambda N: N + 1}
INTEGRAND_XU = {1: lambda N: N, 2: lambda N: 1, 3: lambda N: 0, 4: lambda N: 1,
                5: lambda N: 1}
# Lane-operations per clock per SM of each pipe on GB300, measured by the
# library's instruction-throughput probes (profiles/pipes_gb300.md): the wide
# multiply interleaved with other work, LOP3, FFMA, MUFU.COS/SIN and MUFU.EX2.
PIPE_RATE = {"fma_heavy": 32.0, "alu": 64.0, "fp32": 123.7, "xu_cos": 16.0, "xu_ex2": 32.0}


def pipe_model(gid: int, N: int, prec: int) -> dict:
    """SM-cycles per evaluation that each pipe needs for the algorithmic
    operations of (integrand, N) in an FP32 precision (ops / pipe rate), and
    the issue slots (all operations / 128 lane-slots per clock per SM)."""
    if gid == 0:
        return {}
    xu_rate = PIPE_RATE["xu_ex2"] if gid == 2 else PIPE_RATE["xu_cos"]
    cyc = {"fma_heavy": 4.0 * N / PIPE_RATE["fma_heavy"],
           "alu": 5.0 * N / PIPE_RATE["alu"],
           "fp32": (N + INTEGRAND_FP[gid](N) + ACCUM_OPS[prec]) / PIPE_RATE["fp32"],
           "xu": INTEGRAND_XU[gid](N) / xu_rate,
           "issue": ops_per_eval(gid, N, prec) / 128.0}
    return cyc


def binding_pipe(gid: int, N: int, prec: int, sm_count: int, f_mhz: float,
                 evals_per_s: float) -> dict:
    """The pipe whose algorithmic work per evaluation (pipe_model) allows the
    fewest evaluations per second, that ceiling, and the kernel's share of it."""
    cyc = pipe_model(gid, N, prec)
    if not cyc:
        return {}
    name = max(cyc, key=cyc.get)
    ceil = sm_count * f_mhz * 1e6 / cyc[name]
    return {"pipe": name, "sm_cycles_per_eval": cyc[name], "evals_per_s_at_full_pipe": ceil,
            "frac": evals_per_s / ceil, "source": "algorithmic operations per pipe "
            "(bench.py pipe_model) at the probe-measured pipe rates"}


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ distributed --
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    from paper_1910_01965_gb300 import shard
    shard.barrier()


def max_over_ranks(world, value: float) -> float:
    from paper_1910_01965_gb300 import shard
    return shard.max_over_ranks(value)


# -------------------------------------------------------------- workloads --
def bench_workload(name: str):
    from paper_1910_01965_gb300 import workloads as wl
    if name == "gauss_1e5":   # the same scan on a 10 x 100 x 100 x 1 grid (profiling)
        spec = wl.scan_gauss_1e6()
        spec.lists[0] = spec.lists[0][:10]
        spec.name = "gauss03_N4_P1e5_S2^14_T4"
        return spec
    return {"gauss_1e6": wl.scan_gauss_1e6, "osc_1e4": wl.scan_osc_1e4,
            "cosprod_100": wl.scan_cosprod_100}[name]()


def profile_figures(spec):
    """`key: value` figures of the committed ncu summary of the sampling kernel
    on the Gaussian 10^6-point workload (DRAM bytes of one full-size launch,
    FMA-heavy pipe cycles per evaluation); {} for other workloads, or when the
    kernel sources changed since the counters were taken."""
    from paper_1910_01965_gb300 import build as B
    path = os.path.join(ROOT, "profiles", "scan_kernel_gauss03_N4_fp32k.md")
    if not os.path.exists(path) or spec.integrand_id != 2 or spec.N != 4 or spec.P != 10**6:
        return {}
    figs, src = {}, None
    for line in open(path):
        key, sep, rest = line.partition(":")
        if not sep or " " in key:
            continue
        if key == "kernel_source_stamp":
            src = rest.strip()
        else:
            try:
                figs[key] = float(rest.split()[0])
            except (ValueError, IndexError):
                pass
    return figs if src == B.source_stamp() else {}


# ------------------------------------------------------------- CPU oracle --
def cpu_oracle_run(spec, seconds: float, seed: int = 4242):
    """Time the oracle (as it stands) on a seeded sample of grid points sized
    for about `seconds` of CPU work.  Returns (evals/s, cores, description)."""
    from oracle import oracle
    from paper_1910_01965_gb300 import workloads as wl
    O = oracle.default()
    cores = O.max_threads()
    per_point = spec.trials * spec.samples
    calib = wl.sample_points(spec.P, max(cores, 4), seed=seed + 1)
    t0 = time.perf_counter()
    O.scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                  spec.samples, spec.trials, spec.seed, calib)
    rate = calib.size * per_point / max(time.perf_counter() - t0, 1e-6)
    npts = int(max(cores, min(spec.P, seconds * rate / per_point)))
    pts = wl.sample_points(spec.P, npts, seed=seed)
    t0 = time.perf_counter()
    ref = O.scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                        spec.values, spec.samples, spec.trials, spec.seed, pts,
                        want_sums=True)
    dt = time.perf_counter() - t0
    value = pts.size * per_point / dt
    desc = ("%d of %d grid points (seeded sample), all %d trials x %d samples each: "
            "%.3g evals in %.1f s" % (pts.size, spec.P, spec.trials, spec.samples,
                                      pts.size * per_point, dt))
    return value, cores, desc, pts, ref


def run_reference(args, spec, world, rank):
    if rank != 0:
        return 0
    from paper_1910_01965_gb300 import workloads as wl
    from oracle import oracle
    O = oracle.default()
    cores = O.max_threads()
    per_point = spec.trials * spec.samples
    # size each step for ~args.ref_step_seconds of CPU work
    calib = wl.sample_points(spec.P, max(cores, 4), seed=99)
    t0 = time.perf_counter()
    O.scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                  spec.samples, spec.trials, spec.seed, calib)
    rate = calib.size * per_point / max(time.perf_counter() - t0, 1e-6)
    npts = int(max(cores, min(spec.P, args.ref_step_seconds * rate / per_point)))
    for w in range(args.warmup):
        pts = wl.sample_points(spec.P, npts, seed=1000 + w)
        O.scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                      spec.values, spec.samples, spec.trials, spec.seed, pts)
    total = 0.0
    for k in range(args.steps):
        pts = wl.sample_points(spec.P, npts, seed=2000 + k)
        t0 = time.perf_counter()
        O.scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                      spec.values, spec.samples, spec.trials, spec.seed, pts)
        total += time.perf_counter() - t0
    evals = npts * per_point * args.steps
    value = evals / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(spec.describe(), precision="fp64 (CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: %d seeded grid points of %d, all trials and "
                                   "samples" % (npts, spec.P)},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def accuracy(spec, pts, ref, got):
    """Worst deviation of GPU results from the FP64 oracle over the sampled
    points: scaled by max(|f|, V * RMS(g)) and in standard errors (errw)."""
    V = float(np.prod(np.asarray(spec.hi) - np.asarray(spec.lo)))
    R = V * np.sqrt(np.mean(ref["s2"], axis=1) / spec.samples)
    scale = np.maximum(np.abs(ref["mean"]), R)
    dm = np.abs(got["mean"][pts] - ref["mean"])
    de = np.abs(got["err"][pts] - ref["err"])
    se = ref["errw"]
    return {"points": int(pts.size), "max_dmean_scaled": float(np.max(dm / scale)),
            "max_dmean_stderr": float(np.max(dm / se)),
            "max_derr_stderr": float(np.max(de / se))}


def serving_run(window_s: float, rate: float = 500.0, large_fraction: float = 0.01,
                budget=60 << 30, sample_s: float = 0.25):
    """Open-loop Poisson arrivals through the library's serving loop; every
    request is waited for.  Returns throughput, latency percentiles (all, small
    and large requests) and the queue depth over time (sampled from the
    server's own counters every `sample_s` seconds until the last request is
    done)."""
    import threading
    from paper_1910_01965_gb300 import workloads as wl
    from paper_1910_01965_gb300 import zmc
    arr = wl.serving_poisson(rate=rate, window_s=window_s, large_fraction=large_fraction)
    srv = zmc.Server(budget)
    tickets = []
    depth = []
    stop = threading.Event()

    def sample_depth():
        while not stop.is_set():
            st_ = srv.stats()
            depth.append((round(time.perf_counter() - t0, 3), int(st_.queued), int(st_.active)))
            stop.wait(sample_s)

    t0 = time.perf_counter()
    sampler = threading.Thread(target=sample_depth, daemon=True)
    sampler.start()
    try:
        for a in arr:
            now = time.perf_counter() - t0
            if a.t > now:
                time.sleep(a.t - now)
            sp = a.spec
            tickets.append((srv.submit(sp.integrand_id, sp.N, sp.lo, sp.hi, sp.lengths,
                                       sp.values, sp.samples, sp.trials, sp.seed), a))
        for t, a in tickets:
            srv.wait(t)
        wall = time.perf_counter() - t0
        stop.set()
        sampler.join()
        st = srv.stats()
        lat = {"small": [], "large": []}
        for t, a in tickets:
            lat["large" if a.large else "small"].append(srv.result(t)[1].total_ms)
    finally:
        stop.set()
        srv.close()
    evals = float(sum(a.spec.evals for t, a in tickets))
    outstanding = [q + a_ for _, q, a_ in depth]
    in_window = [q + a_ for t_, q, a_ in depth if t_ <= window_s]
    out = {"arrival_rate_per_s": rate, "window_s": window_s, "large_fraction": large_fraction,
           "requests": len(tickets), "large_requests": len(lat["large"]),
           "offered_evals_per_s": evals / window_s,
           "evals_per_s": evals / wall, "gpu_busy_evals_per_s": st.evals_per_s,
           "utilisation": (evals / window_s) / st.evals_per_s if st.evals_per_s > 0 else 0.0,
           "wall_s": wall, "drain_s": max(0.0, wall - window_s), "steps": st.steps,
           "max_queued": st.max_queued,
           "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mem_peak_bytes": st.mem_peak,
           "budget_bytes": budget,
           "outstanding_max": max(outstanding) if outstanding else 0,
           "outstanding_at_window_end": in_window[-1] if in_window else 0,
           # (seconds since the first arrival, queued, admitted) every sample_s
           "queue_depth": depth}
    for k, v in lat.items():
        if v:
            out["%s_p50_ms" % k] = float(np.percentile(v, 50))
            out["%s_p99_ms" % k] = float(np.percentile(v, 99))
    return out


def sustainable(res) -> bool:
    """A rate is sustainable when the offered work stays below what the GPU
    serves per second of busy time under the same mix (utilisation below 1:
    the queue is stable) and the backlog left at the end of the arrival window
    drains within a quarter of the window (an overloaded queue grows in
    proportion to the window, a stable one stays near the in-flight work)."""
    return res["utilisation"] <= 1.0 and res["drain_s"] <= 0.25 * res["window_s"]


def run_serving_sweep(args, world, rank, local):
    """Open-loop rate sweep of the serving mix: the highest arrival rate whose
    queue stays bounded (see `sustainable`), for the full mix (1 % large) and
    for small requests alone."""
    import torch
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(local)
    zmc.load()
    clocks = ClockSampler(local)
    clocks.start()
    sweeps = {}
    for name, frac, rates, window in (
            ("small_only", 0.0, [50, 100, 125, 150, 175, 200, 250], 4.0),
            ("mix_1pct_large", 0.01, [10, 20, 30, 35, 40, 45, 50, 60], args.serve_window)):
        pts = []
        best = None
        for r in rates:
            res = serving_run(window, float(r), frac)
            ok = sustainable(res)
            pts.append({k: res[k] for k in (
                "arrival_rate_per_s", "requests", "large_requests", "evals_per_s",
                "offered_evals_per_s", "gpu_busy_evals_per_s", "utilisation", "wall_s",
                "drain_s", "p50_ms", "p99_ms", "small_p50_ms", "small_p99_ms", "large_p50_ms",
                "large_p99_ms",
                "outstanding_max", "outstanding_at_window_end", "max_queued")
                if k in res} | {"sustainable": ok})
            if ok:
                best = r
            else:
                break  # higher rates only overload further
        sweeps[name] = {"window_s": window, "large_fraction": frac, "points": pts,
                        "sustainable_rate_per_s": best}
    clk = clocks.stop()
    top = sweeps["mix_1pct_large"]
    line = {"metric": METRIC, "value": max((p["evals_per_s"] for p in top["points"]), default=0.0),
            "unit": "evals/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": sum(p["wall_s"] for s_ in sweeps.values() for p in s_["points"]) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serving rate sweep (open loop, every request waited for)",
                       "criterion": "drain after the window <= 0.25 x window"},
            "sweep": sweeps, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def small_scan_batch(zmc, torch, prec, stream):
    """2048 small scans of the serving mix's kind (the uneven generator with
    samples capped at 2^11 and lists at 8 values): descriptors, outputs and
    the buffers they point into."""
    from paper_1910_01965_gb300 import workloads as wl
    small = [s for s in wl.batch_uneven_256(count=2048, seed=7)]
    for s_ in small:
        s_.samples = int(min(s_.samples, 1 << 11))
        s_.lists = [v[:min(len(v), 8)] for v in s_.lists]
    sd, so, sk = [], [], []
    for sp in small:
        vals = torch.tensor(sp.values, dtype=torch.float64, device="cuda")
        d, k = zmc.make_desc(sp.integrand_id, sp.N, sp.lo, sp.hi, sp.lengths, vals, sp.samples,
                             sp.trials, sp.seed, prec, mem=zmc.ZMC_MEM_DEVICE)
        d.stream = stream.cuda_stream
        m = torch.empty(sp.P, dtype=torch.float64, device="cuda")
        e = torch.empty_like(m)
        o = zmc.zmc_scan_out()
        o.mean, o.err = zmc._ptr(m), zmc._ptr(e)
        sd.append(d)
        so.append(o)
        sk.append((k, vals, m, e))
    return small, sd, so, sk


def run_small_batch_bench(args, world, rank, local):
    """One step = one graph replay of 2048 small scans in one persistent launch
    per precision (the serving mix's typical requests)."""
    import torch
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(local)
    zmc.load()
    prec = zmc.PRECISIONS[args.precision]
    stream = torch.cuda.current_stream()
    small, sd, so, sk = small_scan_batch(zmc, torch, prec, stream)
    evals = float(sum(sp.evals for sp in small))
    ops = float(sum(ops_per_eval(sp.integrand_id, sp.N, prec) * sp.evals for sp in small))
    h = zmc.zmc_batch_create(sd, so, zmc.ZMC_BATCH_GRAPH)
    info = zmc.zmc_batch_info_get(h)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        zmc.zmc_batch_run(h, stream.cuda_stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        zmc.zmc_batch_run(h, stream.cuda_stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    zmc.zmc_batch_destroy(h)
    info_d = zmc.zmc_device_info_get()
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    f_max = json.load(open(peaks)).get("sm_max_mhz") if os.path.exists(peaks) else None
    f_max = f_max or info_d.clock_khz / 1e3
    peak = info_d.sm_count * 128 * f_max * 1e6 / 1e12
    tot = sum(step_ms)
    achieved = ops / (statistics.mean(step_ms) * 1e-3) / 1e12
    line = {"metric": METRIC, "value": evals * args.steps / (tot * 1e-3), "unit": "evals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec else "f64", "data": "synthetic",
            "config": {"workload": "batch_small_2048 (2048 small scans, one persistent launch "
                                   "per precision, CUDA-graph replay)", "scans": len(small),
                       "tiles": int(info.tiles), "evaluations": evals,
                       "precision": args.precision,
                       "l2": "256 MiB buffer written between timed steps"},
            "roofline": {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "batch_kernel (persistent)"},
            "clocks": clk, "gpu_launches": info.launches_per_run * args.steps}
    print(json.dumps(line), flush=True)
    return 0


def run_batch_bench(args, world, rank, local):
    """One step = one run of the 256-scan uneven batch (persistent launch,
    CUDA-graph replay); compared with the same scans as separate launches."""
    import torch
    from paper_1910_01965_gb300 import workloads as wl
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(local)
    zmc.load()
    specs = wl.batch_uneven_256()
    prec = zmc.PRECISIONS[args.precision]
    descs, outs, keep = [], [], []
    for sp in specs:
        vals = torch.tensor(sp.values, dtype=torch.float64, device="cuda")
        d, k = zmc.make_desc(sp.integrand_id, sp.N, sp.lo, sp.hi, sp.lengths, vals, sp.samples,
                             sp.trials, sp.seed, prec, mem=zmc.ZMC_MEM_DEVICE)
        m = torch.empty(sp.P, dtype=torch.float64, device="cuda")
        e = torch.empty_like(m)
        o = zmc.zmc_scan_out()
        o.mean, o.err = zmc._ptr(m), zmc._ptr(e)
        descs.append(d)
        outs.append(o)
        keep.append((k, vals, m, e))
    evals = float(sum(sp.evals for sp in specs))
    ops = float(sum(ops_per_eval(sp.integrand_id, sp.N, prec) * sp.evals for sp in specs))
    stream = torch.cuda.current_stream()

    def one_run_ms():
        hh = zmc.zmc_batch_create(descs, outs, zmc.ZMC_BATCH_GRAPH)
        zmc.zmc_batch_run(hh, stream.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        zmc.zmc_batch_run(hh, stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        zmc.zmc_batch_destroy(hh)
        return a.elapsed_time(b)

    untuned_ms = one_run_ms()
    # the autotuner, once per scan class present (integrand, N, log2 S)
    classes = {}
    for sp, d in zip(specs, descs):
        key = (sp.integrand_id, sp.N, int(np.log2(sp.samples)))
        if key not in classes or sp.evals > classes[key][0].evals:
            classes[key] = (sp, d)
    t_tune = time.perf_counter()
    tuned = 0
    for key, (sp, d) in sorted(classes.items()):
        zmc.zmc_autotune(d, args.tune_ms)
        tuned += 1
    tune_s = time.perf_counter() - t_tune
    h = zmc.zmc_batch_create(descs, outs, zmc.ZMC_BATCH_GRAPH)
    info = zmc.zmc_batch_info_get(h)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        zmc.zmc_batch_run(h, stream.cuda_stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        zmc.zmc_batch_run(h, stream.cuda_stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    zmc.zmc_batch_destroy(h)
    # the same scans, one launch pair each
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for d, o in zip(descs, outs):
        d.stream = stream.cuda_stream
        zmc.zmc_scan_ex(d, o)
    b.record(stream)
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    # Many small scans (the serving mix's typical request): separate launches
    # are overhead-bound there, one persistent launch is not.
    small, sd, so, sk = small_scan_batch(zmc, torch, prec, stream)
    small_evals = float(sum(sp.evals for sp in small))
    hs = zmc.zmc_batch_create(sd, so, zmc.ZMC_BATCH_GRAPH)
    zmc.zmc_batch_run(hs, stream.cuda_stream)
    a.record(stream)
    zmc.zmc_batch_run(hs, stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    small_batch_ms = a.elapsed_time(b)
    zmc.zmc_batch_destroy(hs)
    for d, o in zip(sd, so):
        zmc.zmc_scan_ex(d, o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d, o in zip(sd, so):
        zmc.zmc_scan_ex(d, o)
    torch.cuda.synchronize()
    small_sep_ms = (time.perf_counter() - t0) * 1e3
    info_d = zmc.zmc_device_info_get()
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    f_max = json.load(open(peaks)).get("sm_max_mhz") if os.path.exists(peaks) else None
    f_max = f_max or info_d.clock_khz / 1e3
    peak = info_d.sm_count * 128 * f_max * 1e6 / 1e12
    tot = sum(step_ms)
    achieved = ops / (statistics.mean(step_ms) * 1e-3) / 1e12
    line = {"metric": METRIC, "value": evals * args.steps / (tot * 1e-3), "unit": "evals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec else "f64", "data": "synthetic",
            "config": {"workload": "batch_uneven_256 (256 scans, one persistent launch per "
                                   "precision, CUDA-graph replay)", "scans": len(specs),
                       "tiles": int(info.tiles), "evaluations": evals,
                       "precision": args.precision,
                       "l2": "256 MiB buffer written between timed steps"},
            "roofline": {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "batch_kernel (persistent)"},
            "separate_launches": {"ms": seq_ms, "evals_per_s": evals / (seq_ms * 1e-3),
                                  "launches": 2 * len(specs), "tiles": "autotuned"},
            "small_scans_2048": {"scans": len(small), "evaluations": small_evals,
                                 "batch_ms": small_batch_ms,
                                 "separate_launches_ms": small_sep_ms,
                                 "batch_evals_per_s": small_evals / (small_batch_ms * 1e-3),
                                 "separate_evals_per_s": small_evals / (small_sep_ms * 1e-3)},
            "autotune": {"classes": tuned, "tune_s": tune_s,
                         "untuned_batch_ms": untuned_ms,
                         "untuned_evals_per_s": evals / (untuned_ms * 1e-3)},
            "clocks": clk, "gpu_launches": info.launches_per_run * args.steps}
    print(json.dumps(line), flush=True)
    return 0


def run_serving_bench(args, world, rank, local):
    """The full serving workload: 500 req/s for a 10 s window, 1% large."""
    import torch
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(local)
    zmc.load()
    clocks = ClockSampler(local)
    clocks.start()
    res = serving_run(args.serve_window, args.serve_rate, 0.01)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": res["evals_per_s"], "unit": "evals/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": res["wall_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serving_poisson (open loop, every request waited for)",
                       "arrival_rate_per_s": args.serve_rate, "window_s": args.serve_window},
            "serving": res, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def registry_pipe_table() -> dict:
    """Per-kernel ncu figures of the committed registry profile, keyed
    (integrand, N, precision); {} when the kernel sources changed since the
    counters were taken."""
    from paper_1910_01965_gb300 import build as B
    from paper_1910_01965_gb300 import ncu_table
    path = os.path.join(ROOT, "profiles", "registry_pipes_gb300.md")
    if not os.path.exists(path):
        return {}
    stamp, rows = ncu_table.read_summary(path)
    return rows if stamp == B.source_stamp() else {}


def run_registry(args):
    """Every (integrand, N) of the registry in FP32-Kahan and FP64: one line per
    kernel with its evaluations/s, its roofline on the SM issue peak from the
    algorithmic operations, the binding pipe of the algorithmic per-pipe model,
    and the committed ncu pipe figures of that kernel where they are current.
    ``--registry-scale small`` runs each kernel once on a 10^4-point grid with the
    full-size scan's samples and tiles (the ncu capture of the registry profile)."""
    import torch
    from paper_1910_01965_gb300 import workloads as wl
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(0)
    zmc.load()
    info = zmc.zmc_device_info_get()
    f_max, f_src = _f_max(info)
    small = args.registry_scale == "small"
    gids = [int(g) for g in args.registry_integrands.split(",")]
    Ns = [int(n) for n in args.registry_n.split(",")]
    precs = [p for p in args.registry_precisions.split(",")]
    table = {} if small else registry_pipe_table()
    stream = torch.cuda.current_stream()
    flush = None if small else torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    peak_issue = info.sm_count * 128 * f_max * 1e6 / 1e12
    summary = []
    for gid in gids:
        for N in Ns:
            spec = wl.registry_scan(gid, N)
            full_spec = spec
            if small:
                spec = wl.registry_scan(gid, N, points=10_000)
            vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
            mean = torch.empty(spec.P, dtype=torch.float64, device="cuda")
            err = torch.empty_like(mean)
            for pname in precs:
                p = zmc.PRECISIONS[pname]

                tiles = (0, 0, 0)
                if small:
                    # the full-size scan's tiles: each lane's work has the shape it
                    # has in the timed sweep (same samples, lanes and splits)
                    pf = zmc.scan(full_spec.integrand_id, N, full_spec.lo, full_spec.hi,
                                  full_spec.lengths, full_spec.values, full_spec.samples,
                                  full_spec.trials, full_spec.seed, precision=p,
                                  flags=zmc.ZMC_F_PLAN_ONLY)[1]
                    tiles = (pf.tile_lanes, pf.tile_splits, pf.tile_block)

                def run(count=-1):
                    return zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                           spec.lengths, vals, spec.samples, spec.trials,
                                           spec.seed, mean, err, precision=p,
                                           stream=stream.cuda_stream,
                                           flags=zmc.ZMC_F_TIMINGS, count=count, tiles=tiles)
                if small:
                    run()
                    continue
                run(count=min(spec.P, 64))            # load the kernel, warm the clocks
                steps = args.registry_steps if p != zmc.ZMC_FP64 else 1
                kms, tms = [], []
                for _ in range(steps):
                    flush.zero_()
                    o = run()
                    kms.append(o.kernel_ms)
                    tms.append(o.kernel_ms + o.finalize_ms)
                k_ms = statistics.mean(kms)
                rate = spec.evals / (k_ms * 1e-3)
                line = {"metric": METRIC, "workload": "registry", "integrand": gid,
                        "N": N, "precision": pname, "value": spec.evals / (
                            statistics.mean(tms) * 1e-3), "unit": "evals/s",
                        "kernel_evals_per_s": rate, "kernel_ms": k_ms, "steps": steps,
                        "config": dict(spec.describe(), tiles=[o.tile_lanes, o.tile_splits,
                                                               o.tile_block])}
                if p != zmc.ZMC_FP64:
                    ops = ops_per_eval(gid, N, p)
                    achieved = ops * rate / 1e12
                    line["roofline"] = {"bound": "issue", "achieved": achieved,
                                        "peak": peak_issue, "unit": "Tops/s",
                                        "frac": achieved / peak_issue, "ops_per_eval": ops,
                                        "traffic": None,
                                        "peak_basis": "%d SMs x 128 lane-slots x %.0f MHz (%s)"
                                                      % (info.sm_count, f_max, f_src)}
                    line["binding_pipe"] = binding_pipe(gid, N, p, info.sm_count, f_max, rate)
                m = table.get((gid, N, p))
                if m:
                    meas = {"source": "profiles/registry_pipes_gb300.md (ncu, small grid)"}
                    for pipe in ("heavy", "alu", "lite", "xu", "fp64"):
                        per_sm = pipe == "fp64"     # one FP64 unit per SM, else per SMSP
                        cyc = m.get(pipe + ("_sm_cycles_per_eval" if per_sm
                                            else "_smsp_cycles_per_eval"))
                        if cyc:
                            ceil = info.sm_count * (1 if per_sm else 4) * f_max * 1e6 / cyc
                            meas[pipe] = {"smsp_cycles_per_eval": cyc,
                                          "evals_per_s_at_full_pipe": ceil,
                                          "frac": rate / ceil}
                    meas["registers"] = m.get("registers")
                    meas["inst_per_eval"] = m.get("inst_per_eval")
                    line["measured_pipes"] = meas
                    if p == zmc.ZMC_FP64 and m.get("fp64_sm_cycles_per_eval"):
                        line["roofline"] = {
                            "bound": "fp64", "frac": meas["fp64"]["frac"],
                            "basis": "FP64-pipe cycles per evaluation measured by ncu (the "
                                     "FP64 cos/exp/sin are library routines; their operation "
                                     "counts are not part of the method)"}
                print(json.dumps(line), flush=True)
                summary.append(line)
            del vals, mean, err
    if small:
        print(json.dumps({"workload": "registry", "scale": "small", "kernels": len(gids) *
                          len(Ns) * len(precs)}), flush=True)
        return 0
    fp32 = [l_ for l_ in summary if "binding_pipe" in l_ and l_["binding_pipe"]]
    worst = min(fp32, key=lambda l_: l_["binding_pipe"]["frac"]) if fp32 else None
    print(json.dumps({"workload": "registry", "summary": True, "kernels": len(summary),
                      "worst_fp32_binding_frac": worst and worst["binding_pipe"]["frac"],
                      "worst_fp32_kernel": worst and [worst["integrand"], worst["N"]]}),
          flush=True)
    return 0


def _f_max(info):
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    f_max = json.load(open(peaks)).get("sm_max_mhz") if os.path.exists(peaks) else None
    if f_max:
        return f_max, "sm_max_mhz of MEASURED_PEAKS.json"
    return info.clock_khz / 1e3, "device-reported maximum SM clock"


# Printed in the paper (Table 1, Sec. 3.1; one V100 + Xeon Silver 4110, times in
# seconds, 10^4 samples per point, Python/Numba overhead included).
TABLE1 = {  # (M, N): (delta_r, total_s)
    (1, 1): (0.02512, 0.59343), (1, 2): (0.25034, 0.57227), (1, 3): (1.19949, 0.59330),
    (1, 4): (6.19901, 0.60408), (2, 1): (0.03379, 0.61858), (2, 2): (0.16417, 0.59581),
    (2, 3): (0.87280, 0.61055), (2, 4): (4.12216, 0.62169), (3, 1): (0.02927, 1.26269),
    (3, 2): (0.15052, 1.51221), (3, 3): (0.78052, 1.78097), (3, 4): (4.05029, 2.07094),
    (4, 1): (0.08806, 64.8745), (4, 2): (0.55222, 91.5998), (4, 3): (3.55857, 118.275),
    (4, 4): (22.62904, 147.347)}
# Table 2 (Sec. 3.2): 10^8 points x 10^5 samples, N = 6, 100 batches of 10^6 points;
# GPU evaluation time per batch (s) and the three-node total (s).
TABLE2 = {"V100_per_batch_s": 18.19497, "K40m_per_batch_s": 79.62744,
          "K80_per_batch_s": 89.30734, "cluster_total_s": 721.20234}


def sinsum_closed_form(xsum, N, a):
    """Eq. 2 / Eq. 4 on [0, a]^N: (2 sin(a/2))^N sin(sum x + N a / 2)."""
    return (2.0 * np.sin(a / 2.0)) ** N * np.sin(xsum + N * a / 2.0)


def _grid_xsum(M):
    v = np.arange(100.0)
    xs = np.zeros(1)
    for _ in range(M):
        xs = (xs[:, None] + v[None, :]).ravel()
    return xs


def run_table1(args):
    """Every (M, N) of Table 1 through zmc_scan_ex with host buffers: the scan,
    its host<->device copies and delta r of Eq. 3 (|f| in the denominator)."""
    import torch
    from paper_1910_01965_gb300 import workloads as wl
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(0)
    zmc.load()
    rows = {}
    total_evals, total_s = 0.0, 0.0
    for M in (1, 2, 3, 4):
        for N in (1, 2, 3, 4):
            spec = wl.sinsum_table1(M, N, samples=args.table_samples)
            vals = torch.tensor(spec.values, dtype=torch.float64).pin_memory().numpy()
            mean = torch.empty(spec.P, dtype=torch.float64).pin_memory().numpy()
            err = torch.empty(spec.P, dtype=torch.float64).pin_memory().numpy()
            d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                    vals, spec.samples, spec.trials, spec.seed,
                                    zmc.PRECISIONS[args.precision], flags=zmc.ZMC_F_TIMINGS)
            o = zmc.zmc_scan_out()
            o.mean, o.err = zmc._ptr(mean), zmc._ptr(err)
            zmc.zmc_scan_ex(d, o)            # warm
            t0 = time.perf_counter()
            zmc.zmc_scan_ex(d, o)
            wall = time.perf_counter() - t0
            fth = sinsum_closed_form(_grid_xsum(M), N, 10.0)
            dr = float(np.mean(np.abs(fth - mean) / np.abs(fth)))
            paper_dr, paper_s = TABLE1[(M, N)]
            rows["%d,%d" % (M, N)] = {
                "delta_r": dr, "paper_delta_r": paper_dr, "h2d_ms": o.h2d_ms,
                "kernel_ms": o.kernel_ms + o.finalize_ms, "d2h_ms": o.d2h_ms,
                "total_s": wall, "paper_total_s": paper_s, "speedup_vs_paper": paper_s / wall,
                "evals": spec.evals}
            total_evals += spec.evals
            total_s += wall
    line = {"metric": METRIC, "value": total_evals / total_s, "unit": "evals/s", "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": total_s * 1e3, "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": sum(v[1] for v in TABLE1.values()) / total_s,
            "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": "Table 1 of the paper: sine-sum (Eq. 2) on [0,10]^N, lists "
                                   "{0..99}^M, %d samples, all 16 (M, N)" % args.table_samples,
                       "precision": args.precision, "api": "zmc_scan_ex, pinned host buffers",
                       "vs_baseline": "sum of the paper's total times / ours"},
            "table1": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_table2(args):
    """Table 2's workload on one GPU: 10^8 points x 10^5 samples, N = 6, [0,1]^6,
    then delta r(x1, x2) of Eq. 5 (|f| in the denominator)."""
    import torch
    from paper_1910_01965_gb300 import workloads as wl
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(0)
    zmc.load()
    spec = wl.sinsum_table2(samples=args.table_samples if args.table_samples != 10_000
                            else 100_000)
    vals = torch.tensor(spec.values, dtype=torch.float64).pin_memory().numpy()
    mean = torch.empty(spec.P, dtype=torch.float64).pin_memory().numpy()
    err = torch.empty(spec.P, dtype=torch.float64).pin_memory().numpy()
    d, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed,
                            zmc.PRECISIONS[args.precision], flags=zmc.ZMC_F_TIMINGS)
    o = zmc.zmc_scan_out()
    o.mean, o.err = zmc._ptr(mean), zmc._ptr(err)
    t0 = time.perf_counter()
    zmc.zmc_scan_ex(d, o)
    wall = time.perf_counter() - t0
    fth = sinsum_closed_form(_grid_xsum(4), 6, 1.0)
    rel = (np.abs(fth - mean) / np.abs(fth)).reshape(100, 100, 10000)
    dr12 = rel.mean(axis=2)            # Eq. 5: average over (x3, x4)
    line = {"metric": METRIC, "value": spec.evals / wall, "unit": "evals/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": TABLE2["cluster_total_s"] / wall,
            "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": "Table 2 of the paper: sine-sum (Eq. 4) on [0,1]^6, lists "
                                   "{0..99}^4 (1e8 points), %d samples" % spec.samples,
                       "precision": args.precision, "api": "zmc_scan_ex, pinned host buffers",
                       "vs_baseline": "the paper's three-node total / ours"},
            "table2": {"total_s": wall, "h2d_ms": o.h2d_ms,
                       "kernel_ms": o.kernel_ms + o.finalize_ms, "d2h_ms": o.d2h_ms,
                       "paper": TABLE2,
                       "speedup_vs_V100_100_batches": 100 * TABLE2["V100_per_batch_s"] / wall,
                       "delta_r_x1x2_max": float(dr12.max()),
                       "delta_r_x1x2_median": float(np.median(dr12)),
                       "delta_r_overall": float(rel.mean())}}
    print(json.dumps(line), flush=True)
    return 0


def run_precision_stress(args):
    """The oscillatory scan on [0,2]^6 in FP32, FP32-Kahan and FP64: throughput
    and the worst deviation from the FP64 oracle on seeded grid points."""
    import torch
    from oracle import oracle
    from paper_1910_01965_gb300 import workloads as wl
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(0)
    zmc.load()
    spec = wl.scan_osc_1e4()
    pts = wl.sample_points(spec.P, args.stress_points, seed=31)
    t0 = time.perf_counter()
    ref = oracle.default().scan_points(spec.integrand_id, spec.N, spec.lo, spec.hi,
                                       spec.lengths, spec.values, spec.samples, spec.trials,
                                       spec.seed, pts, want_sums=True)
    oracle_s = time.perf_counter() - t0
    vals = torch.tensor(spec.values, dtype=torch.float64, device="cuda")
    mean = torch.empty(spec.P, dtype=torch.float64, device="cuda")
    err = torch.empty_like(mean)
    out = {}
    for name in ("fp32", "fp32_kahan", "fp64"):
        p = zmc.PRECISIONS[name]
        o = zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, mean, err, precision=p,
                            flags=zmc.ZMC_F_TIMINGS)
        if name != "fp64":
            o = zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                vals, spec.samples, spec.trials, spec.seed, mean, err,
                                precision=p, flags=zmc.ZMC_F_TIMINGS)
        got = {"mean": mean.cpu().numpy(), "err": err.cpu().numpy()}
        out[name] = dict(accuracy(spec, pts, ref, got),
                         evals_per_s=spec.evals / ((o.kernel_ms + o.finalize_ms) * 1e-3),
                         kernel_ms=o.kernel_ms)
    # One thread per (point, trial) summing all 2^20 samples (the paper's
    # thread-per-point layout, Sec. 2): where plain FP32 sums drift.
    for name in ("fp32", "fp32_kahan"):
        o = zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, vals,
                            spec.samples, spec.trials, spec.seed, mean, err,
                            precision=zmc.PRECISIONS[name], tiles=(1, 1, 64),
                            flags=zmc.ZMC_F_TIMINGS)
        got = {"mean": mean.cpu().numpy(), "err": err.cpu().numpy()}
        out[name + "_one_thread_per_unit"] = dict(
            accuracy(spec, pts, ref, got),
            evals_per_s=spec.evals / ((o.kernel_ms + o.finalize_ms) * 1e-3))
    line = {"metric": METRIC, "value": out["fp32_kahan"]["evals_per_s"], "unit": "evals/s",
            "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": out["fp32_kahan"]["kernel_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(spec.describe(), compared_points=int(pts.size),
                           oracle_seconds=oracle_s),
            "precisions": out,
            "fp32_kahan_over_fp64": out["fp32_kahan"]["evals_per_s"] / out["fp64"]["evals_per_s"],
            "kahan_note": "with the planner's tiles each lane sums a few hundred sample "
                          "groups, so plain FP32 and Kahan FP32 lane sums deviate from the "
                          "oracle by the same amount, set by the FP32 evaluation of g; the "
                          "compensation shows only when one thread sums a whole unit "
                          "(the *_one_thread_per_unit entries)"}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- main --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="zmc", choices=["zmc", "reference"])
    ap.add_argument("--workload", default="gauss_1e6")
    ap.add_argument("--precision", default="fp32_kahan", choices=["fp32_kahan", "fp32", "fp64"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=6.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-window", type=float, default=1.0)
    ap.add_argument("--serve-rate", type=float, default=500.0)
    ap.add_argument("--tune-ms", type=int, default=300)
    ap.add_argument("--table-samples", type=int, default=10_000)
    ap.add_argument("--stress-points", type=int, default=48)
    ap.add_argument("--registry-scale", default="full", choices=["full", "small"])
    ap.add_argument("--registry-integrands", default="1,2,3,4,5")
    ap.add_argument("--registry-n", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--registry-precisions", default="fp32_kahan,fp64")
    ap.add_argument("--registry-steps", type=int, default=3)
    ap.add_argument("--tiles", default="",
                    help="lanes,splits,block for the headline scan (default: the planner's)")
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs: the whole grid per rank (own seed), weak scaling")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world, rank, local = dist_setup()
    if args.workload in ("batch_uneven_256", "batch_small_2048"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm times the oracle on the headline workload"}))
            return 0
        if args.workload == "batch_small_2048":
            return run_small_batch_bench(args, world, rank, local)
        return run_batch_bench(args, world, rank, local)
    if args.workload == "registry":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm times the oracle on the headline workload"}))
            return 0
        return run_registry(args)
    if args.workload == "precision_stress":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm times the oracle on the headline workload"}))
            return 0
        return run_precision_stress(args)
    if args.workload in ("table1", "table2"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm times the oracle on the headline workload"}))
            return 0
        return run_table1(args) if args.workload == "table1" else run_table2(args)
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm times the oracle on the headline workload"}))
            return 0
        args.serve_window = 10.0 if args.serve_window == 1.0 else args.serve_window
        return run_serving_bench(args, world, rank, local)
    if args.workload == "serving_sweep":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm times the oracle on the headline workload"}))
            return 0
        args.serve_window = 20.0 if args.serve_window == 1.0 else args.serve_window
        return run_serving_sweep(args, world, rank, local)
    spec = bench_workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, spec, world, rank)

    import torch
    from paper_1910_01965_gb300 import shard
    from paper_1910_01965_gb300 import zmc
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        if args.replicas:
            spec.seed = spec.seed + rank  # an independent problem per rank
    zmc.load()
    info = zmc.zmc_device_info_get()
    prec = zmc.PRECISIONS[args.precision]
    # Several GPUs: each rank scans its contiguous slice of the one grid
    # (strong scaling, no exchange but the host gather), with the tiles the
    # planner picks for the whole grid, so the gathered result equals a
    # one-GPU scan bit for bit; --replicas gives each rank the whole grid
    # under its own seed instead (weak scaling).
    partition = world > 1 and not args.replicas
    first, count = shard.shard_range(spec.P, rank, world) if partition else (0, spec.P)
    req = tuple(int(x) for x in args.tiles.split(",")) if args.tiles else (0, 0, 0)
    if args.workload == "gauss_1e5" and not args.tiles:
        # the profiling cut of the headline grid runs the headline's tiles, so its
        # launch shape per unit is the 10^6-point scan's
        full = bench_workload("gauss_1e6")
        p6 = zmc.scan(full.integrand_id, full.N, full.lo, full.hi, full.lengths, full.values,
                      full.samples, full.trials, full.seed, precision=prec,
                      flags=zmc.ZMC_F_PLAN_ONLY)[1]
        req = (p6.tile_lanes, p6.tile_splits, p6.tile_block)
    plan = zmc.scan(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths, spec.values,
                    spec.samples, spec.trials, spec.seed, precision=prec, tiles=req,
                    flags=zmc.ZMC_F_PLAN_ONLY)[1]
    tiles = (plan.tile_lanes, plan.tile_splits, plan.tile_block) if partition else req
    rank_evals = count * spec.trials * spec.samples

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    vals = torch.tensor(spec.values, dtype=torch.float64, device=dev)
    mean = torch.empty(count, dtype=torch.float64, device=dev)
    err = torch.empty_like(mean)
    errw = torch.empty_like(mean)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step(p=prec, flags=zmc.ZMC_F_TIMINGS):
        return zmc.scan_device(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                               vals, spec.samples, spec.trials, spec.seed, mean, err, errw,
                               precision=p, stream=stream.cuda_stream, flags=flags,
                               first_index=first, count=count, tiles=tiles)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kernel_ms, launches = [], 0
    for k in range(args.steps):
        flush.zero_()                      # L2 flush, outside the timed events
        ev[k][0].record(stream)
        o = step()
        ev[k][1].record(stream)
        kernel_ms.append(o.kernel_ms)      # the sampling kernel, library events
        launches += o.launches
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(world, sum(step_ms))
    job_evals = spec.evals if partition else world * spec.evals
    value = job_evals * args.steps / (total_ms * 1e-3)

    # roofline of the sampling kernel (the dominant one), this rank's launches
    ops = ops_per_eval(spec.integrand_id, spec.N, prec) * rank_evals
    k_ms = statistics.mean(kernel_ms)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    f_max = None
    if os.path.exists(peaks_path):
        f_max = json.load(open(peaks_path)).get("sm_max_mhz")
    f_src = "sm_max_mhz of MEASURED_PEAKS.json"
    if not f_max:
        f_max, f_src = info.clock_khz / 1e3, "device-reported maximum SM clock"
    peak = info.sm_count * 128 * f_max * 1e6 / 1e12   # lane-ops per second, T
    achieved = ops / (k_ms * 1e-3) / 1e12
    figs = profile_figures(spec) if prec == zmc.ZMC_FP32_KAHAN else {}
    prof_src = "profiles/scan_kernel_gauss03_N4_fp32k.md (ncu; read by bench.py, " \
               "valid while the kernel sources are unchanged)"
    roofline = {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": figs.get("traffic_bytes_per_launch"),
                "traffic_source": prof_src if "traffic_bytes_per_launch" in figs else None,
                "kernel": "scan_kernel (sampling)", "kernel_ms": k_ms,
                "ops_per_eval": ops_per_eval(spec.integrand_id, spec.N, prec),
                "peak_basis": "%d SMs x 128 lane-slots x %.0f MHz (%s)" % (
                    info.sm_count, f_max, f_src)}
    kernel_rate = rank_evals / (k_ms * 1e-3)
    if prec != zmc.ZMC_FP64:
        roofline["binding_pipe_model"] = binding_pipe(spec.integrand_id, spec.N, prec,
                                                      info.sm_count, f_max, kernel_rate)
    if "heavy_smsp_cycles_per_eval" in figs:
        # the pipe that binds: each SMSP's FMA-heavy pipe, cycles per evaluation
        # from the committed ncu counters; its ceiling at the same clock
        cyc = figs["heavy_smsp_cycles_per_eval"]
        ceil = info.sm_count * 4 * f_max * 1e6 / cyc
        roofline["binding_pipe"] = {"pipe": "FMA-heavy", "smsp_cycles_per_eval": cyc,
                                    "evals_per_s_at_full_pipe": ceil,
                                    "frac": kernel_rate / ceil, "source": prof_src}

    # end to end through the C ABI with host buffers (pinned); with several
    # GPUs each rank's slice, the slowest rank's time (shard.sharded_scan)
    h_vals = torch.tensor(spec.values, dtype=torch.float64).pin_memory().numpy()
    h_mean = torch.empty(count, dtype=torch.float64).pin_memory().numpy()
    h_err = torch.empty(count, dtype=torch.float64).pin_memory().numpy()
    d_host, keep = zmc.make_desc(spec.integrand_id, spec.N, spec.lo, spec.hi, spec.lengths,
                                 h_vals, spec.samples, spec.trials, spec.seed, prec,
                                 first_index=first, count=count, tiles=tiles)
    o_host = zmc.zmc_scan_out()
    o_host.mean = h_mean.ctypes.data_as(zmc._dp)
    o_host.err = h_err.ctypes.data_as(zmc._dp)
    zmc.zmc_scan_ex(d_host, o_host)        # warm
    e2e_steps = max(3, min(args.steps, 5))

    def e2e_pass(f0, c0):
        for _ in range(e2e_steps):
            zmc.zmc_scan_ex(d_host, o_host)
        return {"mean": h_mean}
    if partition:
        gathered, e2e_s = shard.sharded_scan(spec.P, e2e_pass)
    else:
        barrier(world)
        t0 = time.perf_counter()
        e2e_pass(0, spec.P)
        e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": job_evals * e2e_steps / e2e_s, "unit": "evals/s",
           "h2d_bytes_per_step": int(h_vals.nbytes) * world,
           "d2h_bytes_per_step": int(h_mean.nbytes + h_err.nbytes) * world,
           "steps": e2e_steps, "api": "zmc_scan_ex (ZMC_MEM_HOST, pinned host buffers)"}

    extra = {}
    got = {"mean": mean.cpu().numpy(), "err": err.cpu().numpy()}
    if partition:                          # the whole grid from every rank's slice
        got = {k: shard.gather_slices(v, spec.P) for k, v in got.items()}
        extra["partition"] = {"ranks": world, "slice_points": count,
                              "tiles": list(tiles),
                              "e2e_gather_equals_device": bool(np.array_equal(
                                  gathered["mean"], got["mean"]))}
    got64 = None
    if rank == 0 and not args.no_fp64 and prec != zmc.ZMC_FP64 and not partition:
        step(zmc.ZMC_FP64, zmc.ZMC_F_SYNC)  # warm the FP64 kernel
        o64 = step(zmc.ZMC_FP64)
        got64 = {"mean": mean.cpu().numpy(), "err": err.cpu().numpy()}
        fp64_v = spec.evals / (o64.total_ms * 1e-3)
        extra["fp64_path"] = {"value": fp64_v, "unit": "evals/s", "ms_per_step": o64.total_ms,
                              "kernel_ms": o64.kernel_ms,
                              "fp32_over_fp64": value / world / fp64_v}

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, cores, desc, pts, ref = cpu_oracle_run(spec, args.cpu_seconds)
        cpu = {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": desc}
        extra["accuracy_vs_oracle"] = {args.precision: accuracy(spec, pts, ref, got)}
        if got64 is not None:
            extra["accuracy_vs_oracle"]["fp64"] = accuracy(spec, pts, ref, got64)
    if rank == 0 and not args.no_serve:
        extra["serving"] = serving_run(args.serve_window)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if partition else "weak", "vs_baseline": None,
            "dtype": "f64" if prec == zmc.ZMC_FP64 else "f32",
            "data": "synthetic",
            "config": dict(spec.describe(), precision=args.precision,
                           parallelism=("contiguous slice of the grid per GPU" if partition
                                        else "independent scan per GPU" if world > 1
                                        else "1 GPU"),
                           tiles=[o.tile_lanes, o.tile_splits, o.tile_block],
                           l2="256 MiB buffer written between timed steps"),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
