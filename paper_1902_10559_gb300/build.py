"""Build libsplitsart.so in-tree for sm_103a.

The CUDA translation units are compiled with nvcc, the host C++ with g++, in
parallel. Output: ``paper_1902_10559_gb300/libsplitsart.so``. Objects go to
``paper_1902_10559_gb300/_build/``.

Host code is compiled with ``-ffp-contract=off``, so that the geometry
(Siddon lengths) is bitwise identical on x86_64 and aarch64. The device
tracer (``geometry_gpu.cu``) is compiled with ``-fmad=false`` for the same
reason: it must give the host tracer's bits.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsplitsart.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["api.cu", "fold.cu", "sart.cu", "os_sart.cu", "cgls.cu", "stream.cu", "ring.cu", "direct.cu", "multi.cu", "cnn.cu", "cnn_mma.cu", "geometry_gpu.cu"]
# The device tracer must round like the host tracer: no fused multiply-adds.
CU_FLAGS = {"geometry_gpu.cu": ["-fmad=false"]}
CPP_SOURCES = ["geometry.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsplitsart.so")


def _run(cmd: list[str]) -> None:
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{proc.stdout}\n{proc.stderr}")


def _stale(obj: str, src: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src, *deps])


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile the library if any source is newer than it. Returns the .so path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "splitsart.h"))
    common = ["-std=c++17", "-O3", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC,-ffp-contract=off",
               "--expt-relaxed-constexpr", *CU_FLAGS.get(src, []), "-c", s, "-o", o]
        jobs.append((o, s, cmd))
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        cmd = ["g++", *common, "-fPIC", "-ffp-contract=off", "-pthread",
               "-I", os.path.join(os.path.dirname(nvcc), "..", "include"), "-c", s, "-o", o]
        jobs.append((o, s, cmd))
    todo = [j for j in jobs if force or _stale(j[0], j[1], headers)]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(todo))) as ex:
            for fut in [ex.submit(_run, cmd) for _, _, cmd in todo]:
                fut.result()
    objs = [o for o, _, _ in jobs]
    if force or todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
