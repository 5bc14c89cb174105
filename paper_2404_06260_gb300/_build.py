"""In-tree build of libmor.so (sm_103a CUDA + C++ host code), no CMake.

Each translation unit compiles in parallel to an object under _lib/obj; the shared
library links against the shared CUDA runtime so it shares the process's CUDA state
with PyTorch.  A rebuild happens only when a source or header is newer than the
library (or force=True).
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libmor.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["mor_api.cu", "mor_assembly.cu", "mor_sparse.cu", "mor_dense.cu",
              "mor_reduced.cu", "mor_noalloc.cu", "mor_coarse.cu", "mor_wide.cu",
              "mor_explicit.cu", "mor_tc.cu"]
CPP_SOURCES = ["mor_plan.cpp"]


def _cuda_home() -> str:
    return os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH") or "/usr/local/cuda"


def _nvcc() -> str:
    return os.path.join(_cuda_home(), "bin", "nvcc")


def _inputs():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES]
    files += glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    files += glob.glob(os.path.join(INCLUDE, "*.h"))
    files.append(os.path.abspath(__file__))
    return files


def source_fingerprint() -> str:
    """SHA-256 over the library sources (identifies the kernels a profile was taken on)."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(_inputs()):
        if os.path.abspath(f) == os.path.abspath(__file__):
            continue
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _run(cmd):
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
    return p.stdout + p.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit for sm_103a and link libmor.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(OBJDIR, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-c", os.path.join(CSRC, f), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for f in CPP_SOURCES:
        obj = os.path.join(OBJDIR, f + ".o")
        cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-pthread", "-c",
               os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
    logs = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for out in ex.map(lambda j: _run(j[0]), jobs):
            logs.append(out)
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp] + [o for _, o in jobs] +
         ["-lpthread"])
    os.replace(tmp, LIB)
    if verbose:
        print("".join(logs))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
