"""Build the CUDA library libtlbm.so in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel with nvcc, then linked into one
shared library exporting the C ABI of include/tlbm.h.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtlbm.so")
# the same sources with every kernel access checked against the population
# buffers (TLBM_DEBUG_BOUNDS): a test build, slower
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libtlbm_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
          f"-I{os.path.join(ROOT, 'include')}"]
# translation unit -> extra flags
UNITS = {
    "api.cu": [],
    "step_2d_f32.cu": [],
    "step_2d_f16.cu": [],
    "step_3d_f32.cu": [],
    "step_3d_f16.cu": [],
    "step_fp64.cu": ["--fmad=false"],
    "noalloc.cu": [],
    "step_staged.cu": [],
    "batch.cu": [],
    "batch_staged.cu": [],
    "conv.cu": [],
    "peak.cu": [],
}


def _sources():
    return [os.path.join(CSRC, u) for u in UNITS]


def _deps():
    return glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "tlbm.h"), __file__]


def stale(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libtlbm.so (debug: libtlbm_debug.so with TLBM_DEBUG_BOUNDS)."""
    lib, bdir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and not stale(debug):
        return lib
    os.makedirs(bdir, exist_ok=True)
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(bdir, unit.replace(".cu", ".o"))
        cmd = [NVCC, *ARCH, *COMMON, *extra, *(["-DTLBM_DEBUG_BOUNDS"] if debug else []), "-c",
               os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(unit)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = lib + f".tmp{os.getpid()}"
    link = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
            *objs, "-o", tmp]
    subprocess.run(link, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
