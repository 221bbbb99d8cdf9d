"""The C-ABI library on the CPU: it builds, loads, exports every declared
symbol, and validates descriptors without touching a GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_01965_gb300 import build, zmc
    build.build()
    return zmc


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(zmc_\w+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_entry_points():
    names = declared_functions()
    for n in ["zmc_scan", "zmc_scan_ex", "zmc_last_error", "zmc_validate",
              "zmc_workspace_size", "zmc_stream_words"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIBRARY)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    bound = {s[0] for s in lib.SIGNATURES}
    for n in declared_functions():
        assert n in bound or n.startswith("zmc_server") or n.startswith("zmc_submit") \
            or n in getattr(lib, "EXTRA_SYMBOLS", ()), n


def _desc(lib, **kw):
    args = dict(gid=1, N=2, lo=[0, 0], hi=[1, 1], lengths=[10, 10],
                values=np.linspace(0.5, 5, 20), S=1 << 10, T=3, seed=0)
    args.update(kw)
    return lib.make_desc(args.pop("gid"), args.pop("N"), args.pop("lo"), args.pop("hi"),
                         args.pop("lengths"), args.pop("values"), **args)


@pytest.mark.parametrize("kw,status", [
    ({}, 0),
    ({"N": 3, "lo": [0, 0, 0], "hi": [1, 1, 1]}, 1),           # M != N
    ({"gid": 9}, 7),                                          # unknown id
    ({"lo": [0, 1], "hi": [1, 1]}, 1),                        # empty box side
    ({"lo": [0, float("nan")]}, 1),                           # not finite
    ({"lengths": [10, 0], "values": np.zeros(10)}, 1),        # empty list
    ({"S": 0}, 1),
    ({"T": 0}, 1),
    ({"precision": 7}, 1),
    ({"first_index": 101}, 1),                                # beyond P
    ({"first_index": 90, "count": 11}, 1),                    # slice beyond P
    ({"first_index": 100, "count": 0}, 0),                    # empty slice is valid
    ({"gid": 5, "N": 8, "lo": [0] * 8, "hi": [1] * 8, "S": 2 ** 31}, 1),  # S*N too big
    ({"gid": 5, "N": 8, "lo": [0] * 8, "hi": [1] * 8, "S": 2 ** 31 - 2 ** 17}, 0),  # at the limit
    ({"gid": 5, "N": 8, "lo": [0] * 8, "hi": [1] * 8, "S": 2 ** 31 - 2 ** 17 + 1}, 1),  # past it
    ({"tiles": (3, 1, 256)}, 1),                              # lanes not a power of 2
    ({"tiles": (32, 1, 100)}, 1),                             # block not multiple of 32
    ({"tiles": (64, 1, 32)}, 1),                              # block below 64
])
def test_validation(lib, kw, status):
    d, keep = _desc(lib, **kw)
    assert lib.zmc_validate(d) == status, lib.zmc_last_error()
    if status:
        assert lib.zmc_last_error() != ""


def test_workspace_size_with_explicit_tiles_needs_no_gpu(lib):
    d, keep = _desc(lib, tiles=(32, 4, 256))
    n = lib.zmc_workspace_size(d)
    # 100 points x 3 trials x 4 splits x 16 bytes of partials, plus host staging
    assert n >= 100 * 3 * 4 * 16


def test_chunk_points_bound_the_workspace(lib):
    """With explicit tiles the workspace holds one chunk of partial sums (and,
    for host buffers, two chunks of outputs); chunk_points < 0 is refused."""
    d, keep = _desc(lib, tiles=(32, 4, 256), mem=lib.ZMC_MEM_DEVICE, values=0x1000)
    whole = lib.zmc_workspace_size(d)
    assert whole == 100 * 3 * 4 * 16
    d.chunk_points = 10
    assert lib.zmc_workspace_size(d) == -(-10 * 3 * 4 * 16 // 256) * 256   # 256-byte aligned
    d.chunk_points = -1
    assert lib.zmc_validate(d) == lib.ZMC_EINVAL
    h, keep2 = _desc(lib, tiles=(32, 4, 256))
    one = lib.zmc_workspace_size(h)
    h.chunk_points = 10
    assert lib.zmc_workspace_size(h) < one


def test_scan_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.ZmcError):
        lib.zmc_scan(1, 2, [0, 0], [1, 1], [10, 10], np.linspace(0.5, 5, 20), 64, 2, 0)


def test_integrand_registry(lib):
    names = [lib.zmc_integrand_info_get(i).name.decode() for i in range(lib.ZMC_G_COUNT)]
    assert names == ["const", "cosprod", "gauss03", "poly", "osc01", "sinsum"]
    with pytest.raises(lib.ZmcError):
        lib.zmc_integrand_info_get(lib.ZMC_G_COUNT)


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1910_01965_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(path, errors="replace").read()
            assert "oracle" not in src.lower() or path.endswith("workloads.py"), path


def test_log_level_one_reports_failed_calls(lib):
    """ZMC_LOG=1 writes each failed call's message to stderr (a child process,
    no GPU needed: validation fails before any device work)."""
    import subprocess
    import sys
    code = ("import numpy as np\n"
            "from paper_1910_01965_gb300 import zmc\n"
            "d, k = zmc.make_desc(1, 2, [0, 0], [1, 1], [10, 0], np.zeros(10), 8, 2, 0)\n"
            "print(zmc.zmc_validate(d))\n")
    for level, expect in (("1", True), ("0", False)):
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                           env=dict(os.environ, ZMC_LOG=level), timeout=120)
        assert r.returncode == 0 and r.stdout.strip() == "1", r.stderr[-1000:]
        assert ("[zmc:1]" in r.stderr and "list 1 has length 0" in r.stderr) == expect, r.stderr
