"""Print the instruction-throughput probes of zmc_pipes.h as a table.

    python -m paper_1910_01965_gb300.pipes [iterations]

Each line: operations per SM per clock, whole-GPU operations per second and
the SM clock the probe ran at.  Philox is counted in calls (4 words each).
"""
import json
import sys

from . import zmc


def measure(iterations: int = 4096):
    zmc.load()
    info = zmc.zmc_device_info_get()
    rows = []
    for pipe, name in enumerate(zmc.PIPE_NAMES):
        r = zmc.zmc_pipe_measure(pipe, iterations)
        rows.append({"pipe": name, "ops_per_clk_per_sm": r.ops_per_clk_per_sm,
                     "ops_per_s": r.ops_per_s, "clock_mhz": r.clock_mhz, "ms": r.ms})
    return {"device": info.name.decode(), "sm_count": info.sm_count, "rows": rows}


def main():
    it = int(sys.argv[1]) if len(sys.argv) > 1 else 4096
    res = measure(it)
    print("device %s, %d SMs" % (res["device"], res["sm_count"]))
    print("%-14s %14s %14s %10s %9s" % ("op", "ops/clk/SM", "Gops/s", "MHz", "ms"))
    for r in res["rows"]:
        print("%-14s %14.2f %14.1f %10.0f %9.2f" % (r["pipe"], r["ops_per_clk_per_sm"],
                                                   r["ops_per_s"] / 1e9, r["clock_mhz"],
                                                   r["ms"]))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
