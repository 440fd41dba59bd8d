"""Build the CUDA library in-tree: paper_1705_02043_gb300/_build/libpkifmm.so.

nvcc compiles each translation unit for sm_103a only (parallel), g++ the host
precompute (OpenMP); the shared library links the CUDA runtime statically.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpkifmm.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["api.cu", "tree.cu", "translate.cu", "m2l_tc.cu", "trans_tc.cu", "precompute_dev.cu"]
CPP = ["precompute.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))
    ] + [os.path.join(HERE, "..", "include", "pkifmm.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    jobs = []
    for f in CU:
        o = os.path.join(OUT, f + ".o")
        jobs.append([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
                     "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, f), "-o", o])
    for f in CPP:
        o = os.path.join(OUT, f + ".o")
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", f"-I{CUDA}/include", "-c",
                     os.path.join(CSRC, f), "-o", o])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose:
        for l in logs:
            sys.stdout.write(l)
    objs = [os.path.join(OUT, f + ".o") for f in CU + CPP]
    tmp = LIB + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp", "-cudart", "static"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
