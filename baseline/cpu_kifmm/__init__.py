"""Plain binary64 KIFMM on the host cores (C++/OpenMP), the CPU baseline.

A separate program (``kifmm_cpu.cpp``): uniform octree, U/V lists with
periodic images, check-surface translations with pseudo-inverses (Sec. 2.2,
Sec. 3.1), the triply periodic root operator from an Ewald sum (Algorithm 2).
It shares no code with the GPU library or the oracle; ``bench.py`` times it
beside the GPU run.  Kernels: Laplace (0), Stokes (1); periodic axes 0 or 7.
"""

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kifmm_cpu.cpp")
LIB = os.path.join(HERE, "_build", "libkifmm_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the shared library with g++ (-O3, OpenMP) if it is missing or older than its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-shared", SRC, "-o", tmp], check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.kifmm_cpu_eval.argtypes = [ctypes.c_int] * 4 + [ctypes.c_int64, P, P, P, P, P]
        lib.kifmm_cpu_eval.restype = ctypes.c_int
        lib.kifmm_cpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().kifmm_cpu_threads())


def evaluate(kernel, periodic, p, leaf_max, x, f):
    """Potentials at the points x [N,3] (in [0,1)^3) of densities f [N] or [N,3]
    at the same points.  Returns (u, times, depth): u shaped like f; times =
    (operator setup s, 0 when cached; tree s; evaluation s)."""
    k = 1 if kernel == 0 else 3
    x = np.ascontiguousarray(x, dtype=np.float64)
    fa = np.ascontiguousarray(f, dtype=np.float64).reshape(len(x), k)
    u = np.zeros((len(x), k))
    t = np.zeros(3)
    d = ctypes.c_int(0)
    rc = _load().kifmm_cpu_eval(kernel, periodic, p, leaf_max, len(x), x.ctypes.data, fa.ctypes.data,
                                u.ctypes.data, t.ctypes.data, ctypes.byref(d))
    if rc != 0:
        raise ValueError("kifmm_cpu_eval: bad arguments (kernel, periodicity, p, leaf size or a point outside the cell)")
    return u.reshape(np.shape(f)), t, d.value
