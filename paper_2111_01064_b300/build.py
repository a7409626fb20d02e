"""Build libmbhlike.so in-tree for B300 (sm_103a) with nvcc.

    python -m paper_2111_01064_b300.build [--force] [--verbose]

The library has no dependency on PyTorch; the Python binding loads it through ctypes.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libmbhlike.so")
DEBUG_LIB = os.path.join(HERE, "libmbhlike_debug.so")   # MBH_DEBUG_CHECKS: in-kernel index checks
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every source to an object in parallel (one nvcc per file), then link.
    debug=True builds libmbhlike_debug.so with MBH_DEBUG_CHECKS (in-kernel index checks that
    record into the device status word and skip the access)."""
    lib = DEBUG_LIB if debug else LIB
    if not force and not _stale(lib):
        return lib
    objdir = os.path.join(HERE, "_build_debug" if debug else "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
             "-I", INCLUDE, "--expt-relaxed-constexpr"]
    if debug:
        flags.append("-DMBH_DEBUG_CHECKS")
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    jobs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        jobs.append((obj, subprocess.Popen([NVCC, *flags, "-c", src, "-o", obj])))
    failed = [obj for obj, p in jobs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, f"nvcc ({', '.join(map(os.path.basename, failed))})")
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", lib + ".tmp", *[o for o, _ in jobs], "-lcudart"])
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
