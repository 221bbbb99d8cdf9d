"""The benchmark's reference arm (the oracle on the host cores) prints one
JSON line in the bench contract's shape; runs on CPU in a few seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
         "--warmup", "3", "--ref-step-seconds", "0.2"],
        cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "evals/s" and d["steps"] == 2 and d["warmup"] >= 3
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_other_workloads_say_unavailable_for_the_reference_arm():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
         "--workload", "serving_sweep"], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and "unavailable" in d


def test_sustainability_criterion():
    sys.path.insert(0, ROOT)
    import bench
    ok = {"utilisation": 0.9, "drain_s": 1.0, "window_s": 20.0}
    assert bench.sustainable(ok)
    assert not bench.sustainable(dict(ok, utilisation=1.1))
    assert not bench.sustainable(dict(ok, drain_s=6.0))


def test_pipe_model_of_the_headline_kernel():
    """Gaussian N = 4 in FP32-Kahan: 16 wide multiplies per evaluation
    (20 per Philox call, 0.8 calls) bind at 32 per clock per SM."""
    sys.path.insert(0, ROOT)
    import bench
    cyc = bench.pipe_model(2, 4, 2)
    assert cyc["fma_heavy"] == 16 / 32 and cyc["alu"] == 20 / 64
    assert cyc["issue"] == 59 / 128 and cyc["xu"] == 1 / 32
    b = bench.binding_pipe(2, 4, 2, 152, 2070.0, 4.41e11)
    assert b["pipe"] == "fma_heavy"
    assert abs(b["evals_per_s_at_full_pipe"] - 152 * 2070e6 * 2) < 1
    assert 0.69 < b["frac"] < 0.71
    # cos-product N = 8: still the wide multiplies (1.0) before the XU (0.5)
    assert bench.binding_pipe(1, 8, 2, 152, 2070.0, 2e11)["pipe"] == "fma_heavy"
    assert bench.pipe_model(0, 3, 2) == {}


def test_ncu_table_round_trip(tmp_path):
    """The ncu summariser maps launch names to (integrand, N, precision),
    reads per-metric CSV rows and gives its markdown rows back."""
    sys.path.insert(0, ROOT)
    from paper_1910_01965_gb300 import ncu_table, workloads
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
           '"Metric Value"')
    name = "void zmc::scan_kernel<4, zmc::Gauss32<4>, 2>(zmc::ScanArgs)"
    rows = [hdr]
    vals = {"sm__pipe_fmaheavy_cycles_active.sum": 2e9, "sm__cycles_elapsed.sum": 1e9,
            "launch__registers_per_thread": 72, "smsp__inst_executed.sum": 1.5e9}
    for m, v in vals.items():
        rows.append('"0","1","python","h","%s","1","7","(256, 1, 1)","(9, 1, 1)","0","10.3",'
                    '"Command line profiler metrics","%s","x","%s"' % (name, m, v))
    rows.append('"1","1","python","h","void zmc::finalize_kernel(zmc::FinalizeArgs)","1","7",'
                '"(256, 1, 1)","(9, 1, 1)","0","10.3","s","launch__registers_per_thread","x","30"')
    out = ncu_table.summarise("==PROF== x\n" + "\n".join(rows))
    assert len(out) == 1 and (out[0]["gid"], out[0]["N"], out[0]["prec"]) == (2, 4, 2)
    ev = workloads.registry_scan(2, 4, **ncu_table.SMALL).evals
    assert abs(out[0]["heavy_smsp_cycles_per_eval"] - 2e9 / ev) < 1e-12
    assert abs(out[0]["heavy_busy_pct"] - 50.0) < 1e-9
    assert out[0]["fp64_sm_cycles_per_eval"] != out[0]["fp64_sm_cycles_per_eval"]  # absent: nan
    md = tmp_path / "s.md"
    md.write_text(ncu_table.markdown(out, "cmd", "stamp123"))
    stamp, table = ncu_table.read_summary(str(md))
    assert stamp == "stamp123" and table[(2, 4, 2)]["registers"] == 72
    assert ncu_table.kernel_key("scan_kernel<8, zmc::CosProd64<8>, 0>") == (1, 8, 0)
