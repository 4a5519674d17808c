"""In-tree build of libsps.so for sm_103a (nvcc, no cmake).

Every translation unit under csrc/ is compiled in parallel and linked into
``paper_1811_04165_gb300/libsps.so`` (static CUDA runtime).  Host code is built
without floating-point contraction so the FP64 delay tables do not depend on
the host architecture.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libsps.so")
BUILD_DIR = os.path.join(PKG, "_build")
# The bounds-checked build (-DSPS_BOUNDS_CHECK=1): the de-dispersion passes test
# every staged shared-memory read against its stage and report violations in
# the plan's status word instead of reading (a check build, not the product).
LIB_CHECKED = os.path.join(PKG, "libsps_checked.so")
BUILD_DIR_CHECKED = os.path.join(PKG, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsps.so")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(src: str, verbose: bool, build_dir: str = BUILD_DIR, checked: bool = False) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [_nvcc(), "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", *ARCH,
           "-I", INCLUDE, "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
           "--expt-relaxed-constexpr"]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"] if verbose else []
        cmd += ["-DSPS_BOUNDS_CHECK=1"] if checked else []
    else:
        cmd = [c for c in cmd if c != "-lineinfo"]
        cmd[1:1] = ["-x", "c++"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def build_library(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile csrc/ into libsps.so (with `checked`, the bounds-checked
    libsps_checked.so) if it is missing or older than its sources."""
    lib = LIB_CHECKED if checked else LIB
    build_dir = BUILD_DIR_CHECKED if checked else BUILD_DIR
    if not force and not stale(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, build_dir, checked), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc(), "-shared", "-o", tmp, *objs, *ARCH, "-cudart", "static", "-Xcompiler", "-fPIC", "-ldl"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
