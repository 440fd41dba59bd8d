"""ctypes binding of the C ABI (include/pkifmm.h).  Argument marshalling only:
every step of the evaluation runs in the CUDA library."""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

OK = 0
ERR = {-1: "INVALID_ARG", -2: "OUT_OF_BOX", -3: "NOT_NEUTRAL", -4: "CUDA", -5: "OOM",
       -6: "TIMEOUT", -7: "CACHE", -8: "UNSUPPORTED"}


class PKIFMMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pkifmm error {code} ({ERR.get(code, '?')}): {msg}")
        self.code = code
        self.name = ERR.get(code, "?")


def load_library():
    """Load _build/libpkifmm.so (building it if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("pkifmm CUDA library missing: " + path)
            lib = ctypes.CDLL(path)
            P, i, u, d, i64, c = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double,
                                  ctypes.c_int64, ctypes.c_char)
            lib.pkifmm_plan_create.argtypes = [ctypes.POINTER(P), i, u, P, d, i, i, i, i, i, i, ctypes.c_char_p]
            lib.pkifmm_evaluate.argtypes = [P, i64, P, P, i64, P, P, P]
            lib.pkifmm_evaluate_host.argtypes = [P, i64, P, P, i64, P, P, P]
            lib.pkifmm_evaluate_batched.argtypes = [P, i, P, P, P, P, P, P, P]
            lib.pkifmm_autotune_leaf.argtypes = [P, i, P, P, P, P, P, P, P, i, i, P, P, P]
            lib.pkifmm_plan_set_far_field.argtypes = [P, i]
            lib.pkifmm_last_stage_times.argtypes = [P, P, i]
            lib.pkifmm_tree_stats.argtypes = [P, P, i]
            lib.pkifmm_tree_export.argtypes = [P, P, P, P, P, P, P, P]
            lib.pkifmm_list_export.argtypes = [P, c, P, P, P]
            lib.pkifmm_surface_singular_values.argtypes = [i, i, P]
            lib.pkifmm_backward_error.argtypes = [i, i, P]
            lib.pkifmm_root_operator.argtypes = [i, u, i, i, P]
            lib.pkifmm_root_operator_finite.argtypes = [i, i, i, i, P]
            lib.pkifmm_plan_create_finite.argtypes = [ctypes.POINTER(P), i, i, i, P, d, i, i, i, i, i, i,
                                                      ctypes.c_char_p]
            lib.pkifmm_precompute_operators.argtypes = [i, u, i, i, i, i, P, P, P, P, P, P]
            lib.pkifmm_plan_destroy.argtypes = [P]
            lib.pkifmm_plan_destroy.restype = None
            lib.pkifmm_strerror.argtypes = [i]
            lib.pkifmm_strerror.restype = ctypes.c_char_p
            lib.pkifmm_morton_order_noalloc.argtypes = [i64, P, P, d, u, i, P, P]
            lib.pkifmm_m2l_tensor_core_enabled.argtypes = []
            lib.pkifmm_m2l_rank.argtypes = [P]
            lib.pkifmm_launch_count.argtypes = []
            lib.pkifmm_launch_count.restype = ctypes.c_int64
            lib.pkifmm_last_error_message.argtypes = []
            lib.pkifmm_last_error_message.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _check(rc):
    if rc < 0:
        lib = load_library()
        raise PKIFMMError(rc, lib.pkifmm_last_error_message().decode())
    return rc


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())  # torch tensor (device or host)


PKIFMM_PRECOMPUTE_HOST = 0x100  # OR-ed into precision: Stage 1 on the host

# ---- C-ABI functions, same names ----

def pkifmm_plan_create(kernel, periodic_axes, box_lo, box_len, p, ell, leaf_max, depth_max,
                       precision, nrhs, cache_dir=None):
    lib = load_library()
    h = ctypes.c_void_p()
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    _check(lib.pkifmm_plan_create(ctypes.byref(h), kernel, periodic_axes, _ptr(lo), float(box_len), p, ell,
                                  leaf_max, depth_max, precision, nrhs,
                                  cache_dir.encode() if cache_dir else None))
    return h


def pkifmm_plan_create_finite(kernel, axis, nimg, box_lo, box_len, p, ell, leaf_max, depth_max, precision, nrhs,
                              cache_dir=None):
    lib = load_library()
    h = ctypes.c_void_p()
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    _check(lib.pkifmm_plan_create_finite(ctypes.byref(h), kernel, axis, nimg, _ptr(lo), float(box_len), p, ell,
                                         leaf_max, depth_max, precision, nrhs,
                                         cache_dir.encode() if cache_dir else None))
    return h


def pkifmm_root_operator_finite(kernel, axis, nimg, p):
    kn = (6 * (p - 1) ** 2 + 2) * (1 if kernel == 0 else 3)
    out = np.zeros((kn, kn))
    _check(load_library().pkifmm_root_operator_finite(kernel, axis, nimg, p, _ptr(out)))
    return out


def pkifmm_evaluate(plan, S, src, dens, T, trg, pot, stream=None):
    return _check(load_library().pkifmm_evaluate(plan, S, _ptr(src), _ptr(dens), T, _ptr(trg), _ptr(pot),
                                                 stream))


def pkifmm_evaluate_host(plan, S, src, dens, T, trg, pot, stream=None):
    return _check(load_library().pkifmm_evaluate_host(plan, S, _ptr(src), _ptr(dens), T, _ptr(trg), _ptr(pot),
                                                      stream))


def pkifmm_evaluate_batched(plan, nprob, src_off, trg_off, src, dens, trg, pot, stream=None):
    so = np.ascontiguousarray(src_off, dtype=np.int64)
    to = np.ascontiguousarray(trg_off, dtype=np.int64)
    if so.shape != (nprob + 1,) or to.shape != (nprob + 1,):
        raise ValueError("offsets must have nprob + 1 entries")
    return _check(load_library().pkifmm_evaluate_batched(plan, nprob, _ptr(so), _ptr(to), _ptr(src), _ptr(dens),
                                                         _ptr(trg), _ptr(pot), stream))


def pkifmm_autotune_leaf(plan, nprob, src_off, trg_off, src, dens, trg, pot, candidates, reps=2, stream=None):
    so = np.ascontiguousarray(src_off, dtype=np.int64)
    to = np.ascontiguousarray(trg_off, dtype=np.int64)
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    best = np.zeros(1, dtype=np.int32)
    ms = np.zeros(len(cand))
    _check(load_library().pkifmm_autotune_leaf(plan, nprob, _ptr(so), _ptr(to), _ptr(src), _ptr(dens), _ptr(trg),
                                               _ptr(pot), _ptr(cand), len(cand), reps, _ptr(best), _ptr(ms),
                                               stream))
    return int(best[0]), ms


def pkifmm_plan_set_far_field(plan, mode):
    return _check(load_library().pkifmm_plan_set_far_field(plan, mode))


def pkifmm_last_stage_times(plan):
    out = np.zeros(9)
    _check(load_library().pkifmm_last_stage_times(plan, _ptr(out), 9))
    return out


def pkifmm_tree_stats(plan):
    out = np.zeros(8, dtype=np.int64)
    _check(load_library().pkifmm_tree_stats(plan, _ptr(out), 8))
    return out


def pkifmm_tree_export(plan, S, T):
    nbox = int(pkifmm_tree_stats(plan)[0])
    level = np.zeros(nbox, np.int32)
    pos = np.zeros((nbox, 3), np.int32)
    parent = np.zeros(nbox, np.int32)
    sr = np.zeros((nbox, 2), np.int64)
    tr = np.zeros((nbox, 2), np.int64)
    sp = np.zeros(S, np.int64)
    tp = np.zeros(T, np.int64)
    _check(load_library().pkifmm_tree_export(plan, _ptr(level), _ptr(pos), _ptr(parent), _ptr(sr), _ptr(tr),
                                             _ptr(sp), _ptr(tp)))
    return dict(level=level, pos=pos, parent=parent, src_range=sr, trg_range=tr, src_perm=sp, trg_perm=tp)


def pkifmm_list_export(plan, name):
    lib = load_library()
    nbox = int(pkifmm_tree_stats(plan)[0])
    n = _check(lib.pkifmm_list_export(plan, name.encode(), None, None, None))
    ptr = np.zeros(nbox + 1, np.int64)
    box = np.zeros(max(n, 1), np.int32)
    sh = np.zeros((max(n, 1), 3), np.int8)
    _check(lib.pkifmm_list_export(plan, name.encode(), _ptr(ptr), _ptr(box), _ptr(sh)))
    return ptr, box[:n], sh[:n]


def pkifmm_surface_singular_values(kernel, p):
    n = 6 * (p - 1) ** 2 + 2
    out = np.zeros(n * (1 if kernel == 0 else 3))
    _check(load_library().pkifmm_surface_singular_values(kernel, p, _ptr(out)))
    return out


def pkifmm_backward_error(kernel, p):
    out = np.zeros(1)
    _check(load_library().pkifmm_backward_error(kernel, p, _ptr(out)))
    return float(out[0])


def pkifmm_root_operator(kernel, periodic_axes, p, ell):
    kn = (6 * (p - 1) ** 2 + 2) * (1 if kernel == 0 else 3)
    out = np.zeros((kn, kn))
    _check(load_library().pkifmm_root_operator(kernel, periodic_axes, p, ell, _ptr(out)))
    return out


def pkifmm_precompute_operators(kernel, periodic_axes, p, ell, precision, where, want_ops=True):
    """Stage 1 without a plan on the host (where=0) or device (where=1).

    Returns (S [kn], m2m [8,kn,kn] | None, l2l [8,kn,kn] | None, root [kn,kn] | None, seconds,
    phases [svd_s, m2m_l2l_s, root_s, jacobi_sweeps] of the device build, zeros for the host build)."""
    kn = (6 * (p - 1) ** 2 + 2) * (1 if kernel == 0 else 3)
    S = np.zeros(kn)
    m2m = np.zeros((8, kn, kn)) if want_ops else None
    l2l = np.zeros((8, kn, kn)) if want_ops else None
    root = np.zeros((kn, kn)) if (want_ops and periodic_axes) else None
    sec, ph = np.zeros(1), np.zeros(4)
    _check(load_library().pkifmm_precompute_operators(kernel, periodic_axes, p, ell, precision, where, _ptr(S),
                                                      _ptr(m2m), _ptr(l2l), _ptr(root), _ptr(sec), _ptr(ph)))
    return S, m2m, l2l, root, float(sec[0]), ph


def pkifmm_morton_order_noalloc(n, xyz, box_lo, box_len, periodic_axes, depth, perm, stream=None):
    """Allocation-free stable Morton ordering; xyz [n,3] float64 and perm [n] int32 device tensors."""
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    return _check(load_library().pkifmm_morton_order_noalloc(n, _ptr(xyz), _ptr(lo), float(box_len), periodic_axes,
                                                             depth, _ptr(perm), stream))


def pkifmm_m2l_rank(plan):
    return _check(load_library().pkifmm_m2l_rank(plan))


def pkifmm_plan_destroy(plan):
    if plan:
        load_library().pkifmm_plan_destroy(plan)


def pkifmm_m2l_tensor_core_enabled():
    return int(load_library().pkifmm_m2l_tensor_core_enabled())


def pkifmm_launch_count():
    return int(load_library().pkifmm_launch_count())


def pkifmm_strerror(code):
    return load_library().pkifmm_strerror(code).decode()


class PeriodicKIFMM:
    """Owns a plan; evaluate() passes torch CUDA tensors' device pointers.

    kernel: LAPLACE (charges -> potential), STOKES (forces -> velocity),
    LAPLACE_FIELD (charges -> potential and gradient), STOKES_PRESSURE (forces
    -> velocity and pressure).  periodic_axes: bit 0 = x, 1 = y, 2 = z (0 free,
    7 triply periodic).  Densities [nrhs, S, k], results [nrhs, T, kt]
    (self.k, self.kt)."""

    def __init__(self, kernel, periodic_axes, box_lo=(0.0, 0.0, 0.0), box_len=1.0, p=6, ell=2,
                 leaf_max=64, depth_max=10, precision=0, nrhs=1, cache_dir=None, precompute="device", images=None):
        """p: surface points per edge (accuracy); ell: image layers in the near
        sum; leaf_max: points per leaf (s); precision: FP64 or MIXED; nrhs:
        density vectors evaluated together; cache_dir: Stage 1 operator cache.
        precompute: "device" (Stage 1 in CUDA kernels) or "host" (OpenMP).
        images: None for the periodic sums; an integer N >= 1 for a finite array
        of cells along the single axis of periodic_axes (copies |n| <= N)."""
        if precompute not in ("device", "host"):
            raise ValueError("precompute must be 'device' or 'host'")
        # k: source density components; kt: target components
        self.kernel, self.nrhs = kernel, nrhs
        self.k = 1 if kernel in (0, 2) else 3
        self.kt = {0: 1, 1: 3, 2: 4, 3: 4}.get(kernel, 1)
        self.n = 6 * (p - 1) ** 2 + 2
        self.kn = self.n * self.k
        flags = PKIFMM_PRECOMPUTE_HOST if precompute == "host" else 0
        if images is None:
            self.handle = pkifmm_plan_create(kernel, periodic_axes, box_lo, box_len, p, ell, leaf_max, depth_max,
                                             precision | flags, nrhs, cache_dir)
        else:
            if periodic_axes not in (1, 2, 4):
                raise ValueError("a finite array runs along one axis: periodic_axes 1, 2 or 4")
            self.handle = pkifmm_plan_create_finite(kernel, {1: 0, 2: 1, 4: 2}[periodic_axes], images, box_lo,
                                                    box_len, p, ell, leaf_max, depth_max, precision | flags, nrhs,
                                                    cache_dir)

    def evaluate(self, src, dens, trg, pot=None, stream=None):
        """src [S,3], dens [nrhs,S,k], trg [T,3] float64 CUDA tensors -> pot [nrhs,T,k]."""
        import torch
        S, T = src.shape[0], trg.shape[0]
        for t in (src, dens, trg):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("inputs must be contiguous float64 CUDA tensors")
        if pot is None:
            pot = torch.empty((self.nrhs, T, self.kt), dtype=torch.float64, device=src.device)
        if stream is None:
            stream = torch.cuda.current_stream(src.device).cuda_stream
        pkifmm_evaluate(self.handle, S, src, dens, T, trg, pot, ctypes.c_void_p(stream))
        return pot

    def evaluate_batched(self, src_off, trg_off, src, dens, trg, pot=None, stream=None):
        """Independent problems in one call: problem j owns rows
        src_off[j]:src_off[j+1] of src/dens and trg_off[j]:trg_off[j+1] of trg
        (CUDA tensors as in evaluate; offsets on the host)."""
        import torch
        for t in (src, dens, trg):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("inputs must be contiguous float64 CUDA tensors")
        nprob = len(src_off) - 1
        if pot is None:
            pot = torch.empty((self.nrhs, trg.shape[0], self.kt), dtype=torch.float64, device=src.device)
        if stream is None:
            stream = torch.cuda.current_stream(src.device).cuda_stream
        pkifmm_evaluate_batched(self.handle, nprob, src_off, trg_off, src, dens, trg, pot, ctypes.c_void_p(stream))
        return pot

    def autotune_leaf(self, src_off, trg_off, src, dens, trg, candidates=(16, 24, 32, 48, 64, 96, 128), reps=2,
                      stream=None):
        """Time the batch for each candidate leaf size and keep the fastest;
        returns (best leaf size, per-candidate ms)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(src.device).cuda_stream
        pot = torch.empty((self.nrhs, trg.shape[0], self.kt), dtype=torch.float64, device=src.device)
        best, ms = pkifmm_autotune_leaf(self.handle, len(src_off) - 1, src_off, trg_off, src, dens, trg, pot,
                                        candidates, reps, ctypes.c_void_p(stream))
        self.leaf_max = best
        return best, ms

    def evaluate_host(self, src, dens, trg, pot=None, stream=None):
        """Host arrays in and out (numpy, or CPU torch tensors, e.g. pinned);
        the host<->device copies happen inside the library call."""
        if isinstance(src, np.ndarray):
            src, dens, trg = (np.ascontiguousarray(a, dtype=np.float64) for a in (src, dens, trg))
        if pot is None:
            pot = np.zeros((self.nrhs, trg.shape[0], self.kt))
        pkifmm_evaluate_host(self.handle, src.shape[0], src, dens, trg.shape[0], trg, pot,
                             ctypes.c_void_p(stream) if stream else None)
        return pot

    def set_far_field(self, mode):
        """FAR_L2L (default) or FAR_DIRECT (Algorithm 2 step d)."""
        pkifmm_plan_set_far_field(self.handle, mode)

    def stage_times(self):
        return pkifmm_last_stage_times(self.handle)

    def m2l_rank(self):
        """Dimension of the V-list M2L: kn (dense operators) or the shared basis's r."""
        return pkifmm_m2l_rank(self.handle)

    def tree_stats(self):
        return pkifmm_tree_stats(self.handle)

    def close(self):
        if self.handle:
            pkifmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
