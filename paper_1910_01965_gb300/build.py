"""Build libzmc.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

    python -m paper_1910_01965_gb300.build            # libzmc.so
    python -m paper_1910_01965_gb300.build --debug    # libzmc_debug.so (bounds checks)
    python -m paper_1910_01965_gb300.build --variant NAME -DKNOB=V ...   # tuning variant

Each sampling-kernel row (one precision x one integrand, N = 1..8) is its own
translation unit of zmc_scan_inst.cu, so the objects compile in parallel.
Objects go to paper_1910_01965_gb300/_build/, the library to
paper_1910_01965_gb300/libzmc.so.  A stamp of the sources and flags makes
repeat builds a no-op.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libzmc.so")
# The checking build: the same sources with ZMC_DEBUG=1 (device-side bounds
# checks that record failures instead of accessing out of range).
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libzmc_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I" + os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _units():
    """(output object name, source, extra flags) for every translation unit."""
    units = []
    for prec in range(3):
        for gid in range(6):
            units.append(("scan_p%d_g%d.o" % (prec, gid), "zmc_scan_inst.cu",
                          ["-DZMC_INST_PREC=%d" % prec, "-DZMC_INST_GID=%d" % gid]))
    for prec in range(3):
        units.append(("batch_p%d.o" % prec, "zmc_batch_inst.cu",
                      ["-DZMC_INST_PREC=%d" % prec]))
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        name = os.path.basename(src)
        if name in ("zmc_scan_inst.cu", "zmc_batch_inst.cu"):
            continue
        units.append((name.replace(".cu", ".o"), name, []))
    return units


def _stamp() -> str:
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(CSRC, "*")) +
                   glob.glob(os.path.join(ROOT, "include", "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


# The sources the single-scan sampling kernel is compiled from.
KERNEL_SOURCES = ["zmc_scan_kernel.cuh", "zmc_integrands.cuh", "zmc_philox.cuh",
                  "zmc_internal.h", "zmc_scan_inst.cu"]


def source_stamp() -> str:
    """Hash of the sampling kernel's sources alone (no flags, no machine): a
    profile of that kernel taken on the GPU machine stays valid while this is
    unchanged."""
    h = hashlib.sha256()
    files = [os.path.join(CSRC, f) for f in KERNEL_SOURCES] + \
        sorted(glob.glob(os.path.join(ROOT, "include", "zmc.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def build(force: bool = False, jobs: int = 0, verbose: bool = False,
          extra_flags=(), lib: str = LIB, build_dir: str = BUILD) -> str:
    """Compile and link; ``extra_flags``, ``lib`` and ``build_dir`` build a
    variant (e.g. other -D tuning values) beside the default library."""
    BUILD_ = build_dir
    stamp_file = os.path.join(BUILD_, "stamp")
    stamp = _stamp() + "|" + " ".join(extra_flags)
    if (not force and os.path.exists(lib) and os.path.exists(stamp_file)
            and open(stamp_file).read() == stamp):
        return lib
    os.makedirs(BUILD_, exist_ok=True)
    nvcc = _nvcc()
    units = _units()
    jobs = jobs or min(len(units), max(2, os.cpu_count() or 4))

    def compile_one(u):
        obj, src, flags = u
        cmd = [nvcc, *NVCC_FLAGS, *extra_flags, *flags, "-c",
               os.path.join(CSRC, src), "-o", os.path.join(BUILD_, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (obj, r.stdout, r.stderr))
        if verbose and r.stderr.strip():
            sys.stderr.write("[%s]\n%s\n" % (obj, r.stderr))
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(compile_one, units))
    objs = [os.path.join(BUILD_, u[0]) for u in units]
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-ldl",
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib


def build_debug(force: bool = False) -> str:
    """libzmc_debug.so: every kernel with its ZMC_DEBUG bounds checks."""
    return build(force=force, extra_flags=("-DZMC_DEBUG=1",), lib=LIB_DEBUG,
                 build_dir=BUILD_DEBUG)


def build_variant(name: str, flags) -> str:
    """A library built with extra compiler flags (e.g. -DZMC_CALLS_IN_FLIGHT=8), as
    libzmc_<name>.so beside the default one (its objects in _build_<name>/), so that
    it finds the kernel headers in csrc/ as the default library does; load it with
    ZMC_LIBRARY=<that path>."""
    return build(extra_flags=tuple(flags), lib=os.path.join(PKG, "libzmc_%s.so" % name),
                 build_dir=os.path.join(PKG, "_build_" + name))


if __name__ == "__main__":
    if "--debug" in sys.argv:
        print(build_debug(force="--force" in sys.argv))
    elif "--variant" in sys.argv:
        i = sys.argv.index("--variant")
        print(build_variant(sys.argv[i + 1], [a for a in sys.argv[i + 2:] if a.startswith("-")]))
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
