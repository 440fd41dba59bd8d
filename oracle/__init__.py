"""Oracle: plain, slow, FP64 CPU reference for the periodic N-body sum.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import or run anything here.  The
CUDA library never calls it and shares no code with it.

What it computes (Sec. 2.2, Eq. (pfmmDef)):

    q_t = sum_s sum_{p in P} K(x_t, y_s + p) phi_s,

with the (s, p) term whose source image coincides with x_t excluded, for the
Laplace kernel 1/r and the Stokes velocity kernel
(1/8pi)(I/r + r r^T/r^3) of Eq. (kexamples).  P is the lattice of periodic
vectors of the cubic box [0,L)^3 along the periodic axes.  The sums over P
are made absolutely convergent with the conventions that fix the result
(Sec. 2.2 compatibility conditions; Sec. 3.4 for Stokes TP):

* free space: plain double loop;
* Laplace TP: Ewald, k = 0 removed (requires neutral charges);
* Stokes TP: Hasimoto split, k = 0 removed (zero mean flow; a net force is
  allowed);
* Laplace / Stokes SP: direct symmetric image sum with an Euler-Maclaurin
  tail (requires neutral charges / zero net force);
* Laplace / Stokes DP (x, y periodic, z free): 2D Ewald split, in-plane
  modes by the trapezoid rule in k_z, the k_par = 0 term in closed form
  (requires neutral charges / zero net in-plane force).

Derived quantities (the paper names the Stokes pressure kernel, R^3 -> R,
beside the velocity kernel):

* Laplace field: the gradient of each of the sums above at the target, term
  by term (``laplace_gradient``, ``laplace_field``);
* Stokes pressure p = f.r/(4 pi r^3) (mu = 1), summed as -(1/4 pi) div of the
  periodic Laplace potentials of the three force components
  (``stokes_pressure``; zero net force).

Functions with no closed-form or brute-force pin say so in their docstring
("parity unpinned").
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

LAPLACE = 0
STOKES = 1


def build(force: bool = False) -> str:
    """Compile oracle/ewald.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "ewald.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, l, i, P = ctypes.c_double, ctypes.c_long, ctypes.c_int, ctypes.c_void_p
            lib.orc_free.argtypes = [i, l, P, P, l, P, P]
            lib.orc_laplace_tp.argtypes = [l, P, P, l, P, d, d, d, i, d, P]
            lib.orc_stokes_tp.argtypes = [l, P, P, l, P, d, d, d, i, d, P]
            lib.orc_stokes_tp_beenakker.argtypes = [l, P, P, l, P, d, d, d, i, d, P]
            lib.orc_laplace_sp.argtypes = [l, P, P, l, P, i, d, l, P]
            lib.orc_dp.argtypes = [i, l, P, P, l, P, d, d, d, d, d, P]
            lib.orc_stokes_sp.argtypes = [l, P, P, l, P, i, d, l, P]
            lib.orc_laplace_grad_free.argtypes = [l, P, P, l, P, P]
            lib.orc_laplace_tp_grad.argtypes = [l, P, P, l, P, d, d, d, i, d, P]
            lib.orc_laplace_dp_grad.argtypes = [l, P, P, l, P, d, d, d, d, d, P]
            lib.orc_laplace_sp_grad.argtypes = [l, P, P, l, P, i, d, l, P]
            _lib = lib
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def kdim(kernel: int) -> int:
    return 1 if kernel == LAPLACE else 3


def free_space(kernel: int, src, dens, trg) -> np.ndarray:
    """Free-space direct sum sum_s K(x_t, y_s) phi_s (coincident pairs skipped)."""
    y, x = _c(src), _c(trg)
    phi = _c(dens).reshape(len(y), kdim(kernel))
    out = np.zeros((len(x), kdim(kernel)))
    _load().orc_free(kernel, len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), _ptr(out))
    return out[:, 0] if kernel == LAPLACE else out


def ewald_params(xi: float | None = None, rc: float | None = None, tol_exp: float = 6.2):
    """Splitting parameter and cutoffs for ~1e-15 relative truncation error.

    Real space: xi*rc = 6.2 (erfc(6.2) ~ 5e-19); Fourier: kc = 2*6.5*xi.
    """
    if xi is None and rc is None:
        rc = 1.0
    if xi is None:
        xi = tol_exp / rc
    if rc is None:
        rc = tol_exp / xi
    kc = 13.0 * xi
    mmax = int(np.ceil(kc / (2 * np.pi)))
    return xi, rc, mmax, kc


def laplace_tp(src, q, trg, L: float = 1.0, xi=None, rc=None) -> np.ndarray:
    """Laplace, triply periodic, Ewald (k = 0 removed) at targets trg."""
    xi, rc, mmax, kc = ewald_params(xi, rc)
    y, x, phi = _c(src), _c(trg), _c(q)
    out = np.zeros(len(x))
    _load().orc_laplace_tp(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), L, xi, rc, mmax, kc, _ptr(out))
    return out


def stokes_tp(src, f, trg, L: float = 1.0, xi=None, rc=None) -> np.ndarray:
    """Stokes velocity, triply periodic, Hasimoto Ewald (zero mean flow)."""
    xi, rc, mmax, kc = ewald_params(xi, rc)
    y, x, phi = _c(src), _c(trg), _c(f).reshape(-1, 3)
    out = np.zeros((len(x), 3))
    _load().orc_stokes_tp(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), L, xi, rc, mmax, kc, _ptr(out))
    return out


def stokes_tp_beenakker(src, f, trg, L: float = 1.0, xi=None, rc=None) -> np.ndarray:
    """Stokes TP by the Beenakker split (a second derivation of the same sum,
    used to pin the Hasimoto one)."""
    xi, rc, mmax, kc = ewald_params(xi, rc)
    kc = 15.0 * xi  # the k^4 weight decays more slowly
    mmax = int(np.ceil(kc / (2 * np.pi)))
    y, x, phi = _c(src), _c(trg), _c(f).reshape(-1, 3)
    out = np.zeros((len(x), 3))
    _load().orc_stokes_tp_beenakker(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), L, xi, rc, mmax, kc, _ptr(out))
    return out


def laplace_sp(src, q, trg, axis: int = 0, L: float = 1.0, M: int = 200) -> np.ndarray:
    """Laplace, singly periodic along ``axis``: image sum |n|<=M + Euler-Maclaurin tail."""
    y, x, phi = _c(src), _c(trg), _c(q)
    out = np.zeros(len(x))
    _load().orc_laplace_sp(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), axis, L, M, _ptr(out))
    return out


def stokes_sp(src, f, trg, axis: int = 0, L: float = 1.0, M: int = 200) -> np.ndarray:
    """Stokes, singly periodic along ``axis`` (zero net force required): image
    sum |n|<=M with a pair-independent 1/n regularisation and a closed-form
    Euler-Maclaurin tail."""
    y, x, phi = _c(src), _c(trg), _c(f).reshape(-1, 3)
    out = np.zeros((len(x), 3))
    _load().orc_stokes_sp(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), axis, L, M, _ptr(out))
    return out


def doubly_periodic(kernel: int, src, dens, trg, L: float = 1.0, xi=None, rc=None) -> np.ndarray:
    """Periodic in x and y (period L), free in z: 2D Ewald sum.

    The k_z integral of every in-plane Fourier mode is taken by the trapezoid
    rule with z period H = (z extent of all points)/L + 8, so the aliased
    images sit at least 8 periods away (weight < exp(-2 pi 8)).
    """
    xi, rc, _, kc = ewald_params(xi, rc)
    y, x = _c(src), _c(trg)
    phi = _c(dens).reshape(len(y), kdim(kernel))
    zs = np.concatenate([y[:, 2], x[:, 2]]) if len(y) + len(x) else np.zeros(1)
    H = (zs.max() - zs.min()) / L + 8.0
    out = np.zeros((len(x), kdim(kernel)))
    _load().orc_dp(kernel, len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), L, xi, rc, kc, H, _ptr(out))
    return out[:, 0] if kernel == LAPLACE else out


def laplace_dp(src, q, trg, L: float = 1.0, xi=None, rc=None) -> np.ndarray:
    return doubly_periodic(LAPLACE, src, q, trg, L, xi, rc)


def stokes_dp(src, f, trg, L: float = 1.0, xi=None, rc=None) -> np.ndarray:
    return doubly_periodic(STOKES, src, f, trg, L, xi, rc)


def periodic_sum(kernel: int, periodic_axes: int, src, dens, trg, L: float = 1.0) -> np.ndarray:
    """Dispatch on (kernel, periodicity bitmask: bit0=x, bit1=y, bit2=z).

    Returns [T] for Laplace and [T][3] for Stokes, in the coordinates given
    (box [0,L)^3).
    """
    if periodic_axes == 0:
        return free_space(kernel, src, dens, trg)
    if periodic_axes == 7:
        return laplace_tp(src, dens, trg, L) if kernel == LAPLACE else stokes_tp(src, dens, trg, L)
    if periodic_axes == 3:
        return doubly_periodic(kernel, src, dens, trg, L)
    if periodic_axes in (1, 2, 4):
        ax = {1: 0, 2: 1, 4: 2}[periodic_axes]
        return laplace_sp(src, dens, trg, axis=ax, L=L) if kernel == LAPLACE else stokes_sp(src, dens, trg, ax, L)
    raise NotImplementedError(f"oracle: kernel {kernel} periodicity {periodic_axes}")


def finite_array(kernel: int, axis: int, nimg: int, src, dens, trg, L: float = 1.0) -> np.ndarray:
    """A finite array of cells along ``axis`` (the cell and its copies shifted by
    n L e_axis, |n| <= nimg; the finite-length channel of Sec. 4): the plain sum
    of the free-space kernel over the 2 nimg + 1 copies of the sources.  No
    compatibility condition is needed (the sum is finite)."""
    y = _c(src)
    out = None
    for n in range(-nimg, nimg + 1):
        ys = y.copy()
        ys[:, axis] += n * L
        v = free_space(kernel, ys, dens, trg)
        out = v if out is None else out + v
    return out


def laplace_gradient(periodic_axes: int, src, q, trg, L: float = 1.0, xi=None, rc=None, M: int = 200) -> np.ndarray:
    """Gradient at the targets of the periodic Laplace potential of
    ``periodic_sum(LAPLACE, ...)``: each term of the same sums differentiated
    with respect to the target.  Returns [T][3]."""
    y, x, phi = _c(src), _c(trg), _c(q)
    out = np.zeros((len(x), 3))
    lib = _load()
    if periodic_axes == 0:
        lib.orc_laplace_grad_free(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), _ptr(out))
    elif periodic_axes == 7:
        xi, rc, mmax, kc = ewald_params(xi, rc)
        lib.orc_laplace_tp_grad(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), L, xi, rc, mmax, kc, _ptr(out))
    elif periodic_axes == 3:
        xi, rc, _, kc = ewald_params(xi, rc)
        zs = np.concatenate([y[:, 2], x[:, 2]]) if len(y) + len(x) else np.zeros(1)
        H = (zs.max() - zs.min()) / L + 8.0
        lib.orc_laplace_dp_grad(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), L, xi, rc, kc, H, _ptr(out))
    elif periodic_axes in (1, 2, 4):
        ax = {1: 0, 2: 1, 4: 2}[periodic_axes]
        lib.orc_laplace_sp_grad(len(y), _ptr(y), _ptr(phi), len(x), _ptr(x), ax, L, M, _ptr(out))
    else:
        raise NotImplementedError(f"oracle: Laplace gradient, periodicity {periodic_axes}")
    return out


def laplace_field(periodic_axes: int, src, q, trg, L: float = 1.0) -> np.ndarray:
    """Potential and its gradient at the targets, [T][4] = (phi, d/dx, d/dy, d/dz)."""
    return np.concatenate([periodic_sum(LAPLACE, periodic_axes, src, q, trg, L)[:, None],
                           laplace_gradient(periodic_axes, src, q, trg, L)], axis=1)


def stokes_pressure(periodic_axes: int, src, f, trg, L: float = 1.0) -> np.ndarray:
    """Pressure of the Stokeslets (mu = 1): p = f.r/(4 pi r^3) per source,
    i.e. p = -(1/4 pi) div Phi with Phi_a the Laplace (1/r) potential of the
    charges f_a; periodic sums through the periodic Laplace gradient (zero
    net force makes each f_a neutral).  Returns [T]."""
    f = _c(f).reshape(-1, 3)
    div = sum(laplace_gradient(periodic_axes, src, f[:, a], trg, L)[:, a] for a in range(3))
    return -div / (4.0 * np.pi)


def error_metrics(u, ref) -> dict:
    """Sec. 3.3 error measures, per velocity component: max abs, mean abs, RMS, relative L2."""
    d = (np.asarray(u) - np.asarray(ref)).ravel()
    r = np.asarray(ref).ravel()
    return {
        "max_abs": float(np.max(np.abs(d))) if d.size else 0.0,
        "mean_abs": float(np.mean(np.abs(d))) if d.size else 0.0,
        "rms": float(np.sqrt(np.mean(d * d))) if d.size else 0.0,
        "rel_l2": float(np.linalg.norm(d) / np.linalg.norm(r)) if d.size else 0.0,
    }
