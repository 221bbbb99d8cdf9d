"""Per-kernel pipe figures of the sampling kernels from an ncu CSV.

Reads the CSV that ``ncu --csv --print-units base --metrics <METRICS>`` writes
for the registry sweep (``bench.py --workload registry --registry-scale
small``), maps each captured ``scan_kernel<N, Functor, precision>`` launch to
its (integrand, N, precision) and its evaluations (the sweep's small grids,
rebuilt from ``workloads.registry_scan``), and writes a markdown summary with
one row per kernel: cycles per evaluation on each pipe (FMA-heavy, ALU,
FMA-lite, XU, FP64), warp instructions per evaluation, registers, warps and
issue activity.  ``read_summary`` gives the rows back to the benchmark.

    python -m paper_1910_01965_gb300.ncu_table <ncu.csv> "<command>" > summary.md
"""
from __future__ import annotations

import csv
import io
import re
import sys

METRICS = ["gpu__time_duration.sum", "sm__cycles_elapsed.sum",
           "sm__pipe_fmaheavy_cycles_active.sum", "sm__pipe_alu_cycles_active.sum",
           "sm__pipe_fmalite_cycles_active.sum", "sm__pipe_xu_cycles_active.sum",
           "sm__pipe_fp64_cycles_active.sum", "smsp__inst_executed.sum",
           "launch__registers_per_thread", "sm__warps_active.avg.pct_of_peak_sustained_active",
           "smsp__issue_active.avg.pct_of_peak_sustained_active"]

FUNCTORS = {"Const": 0, "CosProd": 1, "Gauss": 2, "Poly": 3, "Osc": 4, "SinSum": 5}
_NAME = re.compile(r"scan_kernel<\s*(\d+)\s*,\s*(?:zmc::)?([A-Za-z]+?)(32|64)<\s*\d+\s*>\s*,"
                   r"\s*(\d+)\s*>")
PIPES = [("heavy", "sm__pipe_fmaheavy_cycles_active.sum"),
         ("alu", "sm__pipe_alu_cycles_active.sum"),
         ("lite", "sm__pipe_fmalite_cycles_active.sum"),
         ("xu", "sm__pipe_xu_cycles_active.sum"),
         ("fp64", "sm__pipe_fp64_cycles_active.sum")]
SMALL = {"points": 10_000}   # the sweep's small grids (full-size samples and tiles)
# Column suffix of each pipe's cycles per evaluation: SMSP-cycles (summed over
# the four SMSPs of every SM) for the per-SMSP pipes, SM-cycles for FP64.
UNIT = {"heavy": "_smsp_cycles_per_eval", "alu": "_smsp_cycles_per_eval",
        "lite": "_smsp_cycles_per_eval", "xu": "_smsp_cycles_per_eval",
        "fp64": "_sm_cycles_per_eval"}


def _num(v: str) -> float:
    v = v.strip().replace(",", "")
    try:
        return float(v)
    except ValueError:
        return float("nan")


def parse_csv(text: str):
    """[(kernel name, {metric: value})] in launch order, from either ncu's
    per-metric rows (default page) or its one-row-per-launch raw page."""
    lines = [ln for ln in text.splitlines() if ln.startswith('"')]
    rows = list(csv.reader(io.StringIO("\n".join(lines))))
    if not rows:
        return []
    head = rows[0]
    out = []
    if "Metric Name" in head:
        ik, im, iv, iid = (head.index("Kernel Name"), head.index("Metric Name"),
                           head.index("Metric Value"), head.index("ID"))
        by_id = {}
        for r in rows[1:]:
            if len(r) <= max(ik, im, iv, iid):
                continue
            ent = by_id.setdefault(r[iid], (r[ik], {}))
            ent[1][r[im]] = _num(r[iv])
        for key in sorted(by_id, key=lambda k: int(k) if k.isdigit() else 0):
            out.append(by_id[key])
    else:
        ik = head.index("Kernel Name")
        for r in rows[1:]:
            if len(r) != len(head) or not _NAME.search(r[ik]):
                continue
            out.append((r[ik], {h: _num(v) for h, v in zip(head, r)}))
    return out


def kernel_key(name: str):
    """(integrand id, N, precision) of a scan_kernel launch name, else None."""
    m = _NAME.search(name)
    if not m or m.group(2) not in FUNCTORS:
        return None
    return FUNCTORS[m.group(2)], int(m.group(1)), int(m.group(4))


def summarise(text: str) -> list:
    from paper_1910_01965_gb300 import workloads as wl
    rows = []
    for name, met in parse_csv(text):
        key = kernel_key(name)
        if key is None:
            continue
        gid, N, prec = key
        spec = wl.registry_scan(gid, N, **SMALL)
        ev = float(spec.evals)
        row = {"gid": gid, "N": N, "prec": prec, "evals": ev,
               "duration_ms": met.get("gpu__time_duration.sum", float("nan")) * 1e-6,
               "registers": met.get("launch__registers_per_thread"),
               "warps_active_pct": met.get("sm__warps_active.avg.pct_of_peak_sustained_active"),
               "issue_active_pct": met.get("smsp__issue_active.avg.pct_of_peak_sustained_active"),
               "inst_per_eval": 32.0 * met.get("smsp__inst_executed.sum", float("nan")) / ev}
        cyc = met.get("sm__cycles_elapsed.sum", float("nan"))
        for short, metric in PIPES:
            v = met.get(metric, float("nan"))
            # the FP64 unit is one per SM on GB300; the other pipes one per SMSP
            lanes = 1.0 if short == "fp64" else 4.0
            row[short + UNIT[short]] = v / ev
            row[short + "_busy_pct"] = 100.0 * v / (lanes * cyc) if cyc > 0 else float("nan")
        rows.append(row)
    return rows


PREC_NAMES = {0: "fp64", 1: "fp32", 2: "fp32_kahan"}
GID_NAMES = {0: "const", 1: "cosprod", 2: "gauss03", 3: "poly", 4: "osc01", 5: "sinsum"}


def markdown(rows: list, command: str, stamp: str) -> str:
    out = ["# Sampling kernels of the registry: ncu pipe figures per kernel", "",
           "Each row: one `scan_kernel<N, Functor, precision>` launch on the registry sweep's",
           "small grid (about 10^4 points x 4 trials x 2^15 samples, `workloads.registry_scan`,",
           "with the tiles of the full-size sweep's 10^5-point scan).",
           "Cycles per evaluation on a pipe = that pipe's active cycles summed over the GPU /",
           "evaluations: SMSP-cycles for the FMA-heavy, ALU, FMA-lite and XU pipes (one per",
           "SMSP), SM-cycles for FP64 (one unit per SM on GB300).  A pipe busy every cycle would",
           "allow 152 SMs x 4 SMSPs x clock / that figure evaluations per second (152 SMs x clock /",
           "it for FP64); `bench.py --workload registry` prints this ceiling and the kernel's share",
           "of it for every kernel.  Busy % = active cycles / (pipes x elapsed cycles).", "",
           "Command (GB300, clocks not locked; the same command without ncu exited 0 first):", "",
           "    " + command, "",
           "| kernel | regs | warps % | issue % | inst/eval | heavy | alu | lite | xu | fp64 |"
           " heavy % | alu % | xu % | fp64 % |",
           "|---|---|---|---|---|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        key = "g%d_N%d_p%d" % (r["gid"], r["N"], r["prec"])
        out.append("| %s | %d | %.1f | %.1f | %.1f | %.3f | %.3f | %.3f | %.3f | %.3f | %.1f |"
                   " %.1f | %.1f | %.1f |" % (
                       key, int(r["registers"] or 0), r["warps_active_pct"] or 0,
                       r["issue_active_pct"] or 0, r["inst_per_eval"],
                       r["heavy_smsp_cycles_per_eval"], r["alu_smsp_cycles_per_eval"],
                       r["lite_smsp_cycles_per_eval"], r["xu_smsp_cycles_per_eval"],
                       r["fp64_sm_cycles_per_eval"], r["heavy_busy_pct"], r["alu_busy_pct"],
                       r["xu_busy_pct"], r["fp64_busy_pct"]))
    out += ["", "Kernel keys: g<integrand id>_N<dimension>_p<precision> (integrands: " +
            ", ".join("%d %s" % kv for kv in GID_NAMES.items()) + "; precisions: " +
            ", ".join("%d %s" % kv for kv in PREC_NAMES.items()) + ").", "",
            "kernel_source_stamp: " + stamp, ""]
    return "\n".join(out)


def read_summary(path: str):
    """(kernel source stamp, {(gid, N, prec): figures}) of a summary file."""
    stamp, rows = None, {}
    cols = ["registers", "warps_active_pct", "issue_active_pct", "inst_per_eval",
            "heavy_smsp_cycles_per_eval", "alu_smsp_cycles_per_eval",
            "lite_smsp_cycles_per_eval", "xu_smsp_cycles_per_eval",
            "fp64_sm_cycles_per_eval", "heavy_busy_pct", "alu_busy_pct", "xu_busy_pct",
            "fp64_busy_pct"]
    key_re = re.compile(r"^g(\d+)_N(\d+)_p(\d+)$")
    in_table = True          # the figures table comes first; later sections are prose
    for line in open(path):
        if line.startswith("kernel_source_stamp:"):
            stamp = line.split(":", 1)[1].strip()
            continue
        if line.startswith("## "):
            in_table = False
        if not in_table or not line.startswith("| g"):
            continue
        f = [x.strip() for x in line.strip().strip("|").split("|")]
        m = key_re.match(f[0])
        if not m or len(f) != len(cols) + 1:
            continue
        vals = {}
        for c, v in zip(cols, f[1:]):
            vals[c] = _num(v)
        rows[(int(m.group(1)), int(m.group(2)), int(m.group(3)))] = vals
    return stamp, rows


def main(argv):
    from paper_1910_01965_gb300 import build as B
    text = open(argv[1]).read()
    command = argv[2] if len(argv) > 2 else "(command not given)"
    rows = summarise(text)
    rows.sort(key=lambda r: (-r["prec"], r["gid"], r["N"]))
    sys.stdout.write(markdown(rows, command, B.source_stamp()))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
