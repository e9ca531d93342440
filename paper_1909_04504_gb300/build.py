"""Builds the CUDA library ``_build/libsph_gb300.so`` for sm_103a with nvcc.

Each translation unit compiles in parallel; the objects link into one shared library
with the C ABI of ``include/sph.h``. No CMake, one -gencode, a minute or less.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsph_gb300.so")
# the pair passes and the persistent step: one translation unit per pair-loop precision and
# tile shape, the longest compiles first
UNITS = [f"{k}_{p}_t{t}.cu" for k in ("fused", "pairs") for p in ("f32", "f64") for t in (1, 2, 4, 8)]
# the per-phase kernels whose bodies the persistent step shares
SAME_ROUNDING = ["nnps.cu", "batch.cu", "walls.cu"]
SOURCES = UNITS + ["capi.cu", "nnps.cu", "pairs.cu", "fused.cu", "octree.cu", "adjoint.cu", "batch.cu",
                   "noalloc.cu", "walls.cu", "pec.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "sph.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "-I", CSRC, "--expt-relaxed-constexpr", "-Xcompiler", "-Wall"]
    if ptxas_verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        # the pair passes come in a single-problem and a batch instantiation, and the
        # persistent step repeats the bodies of the per-phase kernels: all of them must round
        # alike, so no multiply-add is fused unless the source asks for it (fma_rn) and no
        # two instantiations can differ in which products they fuse
        extra = ["-fmad=false"] if src in UNITS + SAME_ROUNDING else []
        cmd = [cc] + flags + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or ptxas_verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"nvcc failed on {src}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc link failed")
    os.replace(tmp, LIB)
    for o in objs:  # the library holds everything; the objects only take space
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
