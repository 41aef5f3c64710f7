"""Build libstk.so (the CUDA scorer, sm_103a) in-tree with nvcc."""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libstk.so")
DEBUG_LIB = os.path.join(HERE, "libstk_debug.so")   # STK_DEBUG_BOUNDS: checked gathers, canaries
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
    "--expt-relaxed-constexpr",
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(ROOT, "include", "stk.h"), os.path.abspath(__file__)]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def _build_one(lib: str, objdir: str, defines, verbose: bool, ptxas_v: bool):
    os.makedirs(objdir, exist_ok=True)
    objs, cmds = [], []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [NVCC] + NVCC_FLAGS + list(defines) + ["-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        if ptxas_v:
            cmd += ["-Xptxas", "-v"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        cmds.append(cmd)
        objs.append(obj)
    return cmds, objs


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, debug: bool = True) -> str:
    """Compile every .cu under csrc/ into libstk.so (shared, C ABI exported) and,
    with debug, the bounds-checked libstk_debug.so (-DSTK_DEBUG_BOUNDS)."""
    jobs = []   # (lib, cmds, objs)
    if force or stale(LIB):
        jobs.append((LIB,) + _build_one(LIB, os.path.join(HERE, "_build"), [], verbose, ptxas_v))
    if debug and (force or stale(DEBUG_LIB)):
        jobs.append((DEBUG_LIB,) + _build_one(DEBUG_LIB, os.path.join(HERE, "_build_debug"), ["-DSTK_DEBUG_BOUNDS"],
                                              verbose, ptxas_v))
    if not jobs:
        return LIB
    cmds = [c for _, cs, _ in jobs for c in cs]
    # the translation units are independent: compile them side by side
    workers = max(1, min(len(cmds), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as pool:
        for f in [pool.submit(subprocess.run, cmd, check=True) for cmd in cmds]:
            f.result()
    for lib, _, objs in jobs:
        tmp = lib + ".tmp.%d" % os.getpid()
        subprocess.run([NVCC, "-shared", "-cudart", "static", "-o", tmp] + objs, check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True, ptxas_v="-v" in sys.argv))
