"""Build librmsbr.so in-tree with nvcc for sm_103a.

Every .cu file under csrc/ is compiled separately (the tracer with
-fmad=false, so that forward and adjoint take bit-identical decisions) and
linked into one shared library against the shared CUDA runtime.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "librmsbr.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
# trace.cu: no contraction (forward, record and adjoint instantiations round
# every choice-steering operation alike).  Both kernels use approximate
# division and square root (a few ulp); the slab tests' reciprocals stay
# correctly rounded through __frcp_rn, which their robustness bound assumes.
PER_FILE = {"trace.cu": ["-fmad=false", "-prec-div=false", "-prec-sqrt=false"], "diffraction.cu": ["-fmad=false", "-prec-div=false", "-prec-sqrt=false"]}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "rmsbr.h"), __file__]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    for src in _sources():
        name = os.path.basename(src)
        obj = os.path.join(BUILD, name + ".o")
        cmd = [NVCC, *ARCH, *COMMON, *PER_FILE.get(name, []), "-c", src, "-o", obj]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        objs.append(obj)
    link = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs,
            "-Xlinker", f"-rpath,{CUDA_HOME}/lib64"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    subprocess.check_call(link)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
