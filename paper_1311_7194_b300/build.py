"""Build libtsdf.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc.

    python -m paper_1311_7194_b300.build [--force] [--verbose] [--debug]

Objects go to ``paper_1311_7194_b300/_build/``; the shared library is written
next to this file so that it travels with the source tree. ``--debug`` builds
libtsdf_debug.so instead: the same sources with TSDF_DEBUG defined, whose
kernels check their table, pool and map indices on the device and report a
failed check as TSDF_ERR_BOUNDS (objects in ``_build/debug/``).
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtsdf.so")
LIB_DEBUG = os.path.join(HERE, "libtsdf_debug.so")
SOURCES = ["tsdf_volume.cu", "tsdf_alloc.cu", "tsdf_integrate.cu", "tsdf_raycast.cu", "tsdf_noalloc.cu", "tsdf_graph.cu",
           "tsdf_autotune.cu", "tsdf_mlp.cu", "tsdf_icp.cu", "tsdf_mesh.cu", "tsdf_evict.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# No FMA contraction: every fused multiply-add is written out (__fmaf_rn), so the
# allocation arithmetic and the Kalman update are the same op sequence wherever
# they are inlined. Host code (pose preparation) is plain IEEE double.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", INCLUDE, "-I", CSRC]
# The raycast has no bit-exact contract with the oracle (its bar is 0.1 voxel),
# and its two kernels share every expression, so the compiler may fuse its
# multiply-adds: measured 1 % faster, results of the two kernels still equal.
PER_FILE_FLAGS = {"tsdf_raycast.cu": {"-fmad=false": "-fmad=true"}}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtsdf.so")


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "tsdf_internal.cuh"), os.path.join(CSRC, "tsdf_storage.cuh"),
              os.path.join(CSRC, "tsdf_mlp.cuh"),
              os.path.join(INCLUDE, "tsdf.h")]
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    obj_dir = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (["-DTSDF_DEBUG"] if debug else [])

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        f = [PER_FILE_FLAGS.get(src, {}).get(x, x) for x in flags]
        cmd = [cc, *ARCH, *f, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
