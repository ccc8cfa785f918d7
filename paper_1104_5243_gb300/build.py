"""Build libbp1104.so in-tree: nvcc for sm_103a, one object per .cu file
compiled in parallel, then one shared library (CUDA runtime linked
statically, no PyTorch types anywhere in the ABI).  build_f64() builds the
separate float64 gradient-check library libbp1104_f64.so from csrc/check/
(test support only; include/bp1104_f64.h)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbp1104.so")
LIB_F64 = os.path.join(BUILD, "libbp1104_f64.so")
CHECK = os.path.join(CSRC, "check")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-Wall", "-I", INCLUDE]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hdrs


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False) -> str:
    """Compile every .cu under csrc/ and link libbp1104.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    newest_dep = max(os.path.getmtime(p) for p in srcs + _deps() + [__file__])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest_dep:
        return LIB
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc()] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def build_f64(force: bool = False) -> str:
    """Compile the float64 gradient-check library (csrc/check/*.cu, which
    instantiates the direct kernel templates of csrc/bp_direct.cuh in
    double); returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(os.path.join(CHECK, f) for f in os.listdir(CHECK) if f.endswith(".cu"))
    newest_dep = max(os.path.getmtime(p) for p in srcs + _deps() + [__file__])
    if not force and os.path.exists(LIB_F64) and os.path.getmtime(LIB_F64) >= newest_dep:
        return LIB_F64
    tmp = LIB_F64 + f".{os.getpid()}.tmp"
    cmd = [nvcc()] + NVCC_FLAGS + ["-shared", "-o", tmp] + srcs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for the float64 check library:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_F64)
    return LIB_F64


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv, force="-f" in sys.argv))
