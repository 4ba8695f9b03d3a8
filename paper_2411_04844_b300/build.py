"""Build libdgr.so in-tree for sm_103a with nvcc (no torch involved).

    python -m paper_2411_04844_b300.build [--force] [--verbose]

Flags: -O3, -lineinfo, no --use_fast_math (the FP32 footprint sequence and
the IEEE divisions of the projector rely on default rounding).

    python -m paper_2411_04844_b300.build --checked

builds libdgr_checked.so with -DDGR_CHECK_BOUNDS: the walks', the FVR
adjoint's and the voxelizer's global accesses test their indices and report
an index outside its buffer as DGR_STATUS_BOUNDS instead of faulting (the
library the binding loads when DGR_CHECK_BOUNDS=1 is set).
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libdgr.so")
LIB_CHECKED = os.path.join(LIBDIR, "libdgr_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    objdir = os.path.join(LIBDIR, "checked") if checked else LIBDIR
    os.makedirs(objdir, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    objs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               *(["-DDGR_CHECK_BOUNDS"] if checked else []), "-I", INCLUDE, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
        objs.append(obj)
    tmp = lib + ".tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, checked="--checked" in sys.argv))
