"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer.

libzmc.so is rebuilt with its host code instrumented (-fsanitize=address and
-fsanitize=undefined, no recovery) and the CPU tests of its C ABI run against
it in a child process: descriptor validation, workspace sizing and chunk
layouts, the registry, the log levels and the run-time compilation of user
integrands (NVRTC), none of which needs a GPU.  Any out-of-bounds access, use
after free, overflow or other undefined behaviour in that host code fails the
test.  The device code is checked by the ZMC_DEBUG build on the GPU instead.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _runtime(name):
    p = subprocess.run(["gcc", "-print-file-name=%s" % name], capture_output=True,
                       text=True).stdout.strip()
    return p if p and os.path.isabs(p) and os.path.exists(p) else None


def test_host_code_runs_clean_under_sanitizers():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("gcc's sanitizer runtimes are not installed")
    from paper_1910_01965_gb300 import build
    flags = ("-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
             "-Xcompiler", "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize-recover=all")
    lib = build.build_variant("hostsan", flags)
    env = dict(os.environ, ZMC_LIBRARY=lib, LD_PRELOAD=asan + ":" + ubsan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_abi_cpu.py"),
                        os.path.join(HERE, "test_user_integrand_cpu.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, \
        r.stderr[-3000:]
    assert " passed" in r.stdout and "failed" not in r.stdout, r.stdout[-2000:]
