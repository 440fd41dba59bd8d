"""Host-side checks of the CUDA library (no GPU needed): the shared object
loads and exports every declared entry point, and the operator precompute
(surfaces, SVD, root far-field operator) agrees with the paper's tables and
with the oracle."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1705_02043_gb300 as pk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _declared():
    hdr = open(os.path.join(ROOT, "include", "pkifmm.h")).read()
    return sorted(set(re.findall(r"\b(pkifmm_[a-z_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    lib = pk.load_library()
    names = _declared()
    assert "pkifmm_plan_create" in names and "pkifmm_evaluate" in names
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def _table_cond():
    rows = []
    for line in open(os.path.join(GOLDEN, "table_cond.txt")):
        if line.strip() and not line.startswith("#"):
            k, p, kappa, rank, dim = line.split()
            rows.append((0 if k == "laplace" else 1, int(p), float(kappa), int(rank), int(dim)))
    return rows


@pytest.mark.parametrize("row", [r for r in _table_cond() if r[2] < 1e15], ids=lambda r: f"k{r[0]}p{r[1]}")
def test_surface_conditioning_matches_table_1(row):
    """Table 1: kappa(A) and numerical rank of the check-to-equivalent matrix
    pin the surface geometry (edges 1.05 / 2.95, p points per edge) and SVD."""
    kernel, p, kappa, rank, dim = row
    s = pk.pkifmm_surface_singular_values(kernel, p)
    assert s.size == dim
    assert np.all(np.diff(s) <= 0)
    assert s[0] / s[-1] == pytest.approx(kappa, rel=0.1)
    assert int(np.sum(s > 2.0 ** -52 * s[0] * dim)) == rank


@pytest.mark.parametrize("kernel,p", [(0, 8), (1, 6)])
def test_backward_stable_solve(kernel, p):
    """Sec. 3.1 / Appendix B: applying V (S+ (U^T b)) keeps the backward error
    near machine precision (the paper reports ~1e-13 at Stokes p = 16)."""
    assert pk.pkifmm_backward_error(kernel, p) < 1e-12


def _surface(p, half=0.525):
    g = np.array([[-1 + 2 * i / (p - 1), -1 + 2 * j / (p - 1), -1 + 2 * k / (p - 1)]
                  for i in range(p) for j in range(p) for k in range(p)
                  if i in (0, p - 1) or j in (0, p - 1) or k in (0, p - 1)])
    return half * g + 0.5


def _near_sum(kernel, x, y, f, periodic):
    """sum over images |p|_inf <= 1 (periodic axes) of K(x, y + p) f, skipping r = 0."""
    rng = [(-1, 0, 1) if periodic >> a & 1 else (0,) for a in range(3)]
    near = np.array([[a, b, c] for a in rng[0] for b in rng[1] for c in rng[2]], float)
    d = x[:, None, :] - y[None, None, :] - near[None]
    r = np.linalg.norm(d, axis=-1)
    rs = np.where(r > 0, r, 1.0)
    if kernel == 0:
        return np.where(r > 0, f / rs, 0.0).sum(1)
    u = (f[None, None, :] / rs[..., None] + d * ((d @ f) / rs ** 3)[..., None]) / (8 * np.pi)
    return np.where((r > 0)[..., None], u, 0.0).sum(1)


@pytest.mark.parametrize("kernel", [0, 1])
def test_root_operator_matches_oracle_tp(kernel):
    """Root operator column j = K^P(x_i - y_j) minus the 27 nearest images,
    with K^P from the oracle's Ewald sum (an independent implementation)."""
    p = 4
    x = _surface(p)
    M = pk.pkifmm_root_operator(kernel, 7, p, 2)
    k = 1 if kernel == 0 else 3
    for j in (0, 9, len(x) - 1):
        for b in range(k):
            f = np.zeros(3)
            f[b] = 1.0
            if kernel == 0:
                kp = oracle.laplace_tp(x[j:j + 1], np.array([1.0]), x)
                ref = kp - _near_sum(0, x, x[j], 1.0, 7)
            else:
                kp = oracle.stokes_tp(x[j:j + 1], f[None], x)
                ref = (kp - _near_sum(1, x, x[j], f, 7)).ravel()
            assert np.max(np.abs(M[:, k * j + b] - ref)) < 1e-12 * max(1.0, np.abs(ref).max())


def test_root_operator_matches_oracle_sp():
    """Singly periodic Laplace: compare neutral combinations (column
    differences), since the two sides may regularise the divergent constant
    differently; it cancels for neutral charges."""
    p = 4
    x = _surface(p)
    M = pk.pkifmm_root_operator(0, 4, p, 2)
    for j, jj in ((0, 5), (3, 20), (11, 40)):
        ref = oracle.laplace_sp(x[[j, jj]], np.array([1.0, -1.0]), x, axis=2)
        ref -= _near_sum(0, x, x[j], 1.0, 4) - _near_sum(0, x, x[jj], 1.0, 4)
        assert np.max(np.abs(M[:, j] - M[:, jj] - ref)) < 1e-12


@pytest.mark.parametrize("kernel", [0, 1])
def test_root_operator_matches_oracle_dp(kernel):
    """Doubly periodic (x, y): the library sums the in-plane Fourier modes in
    closed form, the oracle by the trapezoid rule in k_z.  Compare neutral
    combinations (column differences): the sheet term's constant cancels."""
    p = 4
    x = _surface(p)
    M = pk.pkifmm_root_operator(kernel, 3, p, 2)
    k = 1 if kernel == 0 else 3
    for j, jj in ((0, 5), (3, 20), (11, len(x) - 1)):
        for b in range(k):
            f = np.zeros(3)
            f[b] = 1.0
            if kernel == 0:
                ref = oracle.laplace_dp(x[[j, jj]], np.array([1.0, -1.0]), x)
                ref = ref - (_near_sum(0, x, x[j], 1.0, 3) - _near_sum(0, x, x[jj], 1.0, 3))
            else:
                ref = oracle.stokes_dp(x[[j, jj]], np.stack([f, -f]), x)
                ref = (ref - (_near_sum(1, x, x[j], f, 3) - _near_sum(1, x, x[jj], f, 3))).ravel()
            got = M[:, k * j + b] - M[:, k * jj + b]
            assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("axis", [0, 2])
def test_root_operator_matches_oracle_sp_stokes(axis):
    """Singly periodic Stokes: neutral combinations (column differences),
    library (explicit n <= 512 + Euler-Maclaurin) vs oracle."""
    p = 4
    x = _surface(p)
    per = 1 << axis
    M = pk.pkifmm_root_operator(1, per, p, 2)
    for j, jj in ((0, 5), (3, 20), (11, len(x) - 1)):
        for b in range(3):
            f = np.zeros(3)
            f[b] = 1.0
            ref = oracle.stokes_sp(x[[j, jj]], np.stack([f, -f]), x, axis=axis)
            ref = (ref - (_near_sum(1, x, x[j], f, per) - _near_sum(1, x, x[jj], f, per))).ravel()
            got = M[:, 3 * j + b] - M[:, 3 * jj + b]
            assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("kernel,periodic", [(0, 7), (1, 7), (0, 1), (1, 2), (0, 3), (1, 3)])
def test_root_operator_independent_of_ell(kernel, periodic):
    """Folding layers 2..ell back in makes the operator independent of ell
    (Sec. 3.6: the results do not depend on ell)."""
    M1 = pk.pkifmm_root_operator(kernel, periodic, 4, 1)
    for ell in (2, 3):
        M = pk.pkifmm_root_operator(kernel, periodic, 4, ell)
        assert np.max(np.abs(M - M1)) < 1e-12 * np.abs(M1).max()
    assert np.allclose(M1, M1.T, atol=1e-13 * np.abs(M1).max())  # symmetric kernels


def test_unsupported_and_invalid_arguments():
    with pytest.raises(pk.PKIFMMError) as e:
        pk.pkifmm_root_operator(1, 5, 4, 2)  # built for (x, y); plans run (x, z), (y, z) in a permuted frame
    assert e.value.name == "UNSUPPORTED"
    with pytest.raises(pk.PKIFMMError) as e:
        pk.pkifmm_root_operator(0, 7, 1, 2)
    assert e.value.name == "INVALID_ARG"
    assert pk.pkifmm_strerror(-3).startswith("compatibility")


def test_precompute_entry_host_build():
    # the plan-free Stage 1 entry point on the host: the same root operator as
    # pkifmm_root_operator, singular values of Table 1's matrix, argument checks
    from paper_1705_02043_gb300 import _binding as b
    S, m2m, l2l, root, sec, _ = b.pkifmm_precompute_operators(1, 7, 5, 2, pk.FP64, 0)
    assert sec > 0 and m2m.shape == (8, 294, 294) and l2l.shape == (8, 294, 294)
    np.testing.assert_array_equal(root, b.pkifmm_root_operator(1, 7, 5, 2))
    ref = np.zeros(294)
    pk.load_library().pkifmm_surface_singular_values(1, 5, ref.ctypes.data_as(ctypes.c_void_p))
    assert np.all(np.diff(S) <= 0) and np.abs(S - ref).max() <= 1e-13 * S[0]
    S0, _, _, root0, _, _ = b.pkifmm_precompute_operators(0, 0, 5, 2, pk.FP64, 0, want_ops=False)
    assert root0 is None and len(S0) == 98
    with pytest.raises(pk.PKIFMMError):
        b.pkifmm_precompute_operators(0, 7, 5, 2, pk.FP64, 2)
    with pytest.raises(pk.PKIFMMError):
        b.pkifmm_precompute_operators(0, 5, 5, 2, pk.FP64, 0)


@pytest.mark.parametrize("kernel", [0, 1])
def test_finite_array_root_operator(kernel):
    # a finite array of cells: the root operator is the free-space kernel from
    # the root's upward equivalent surface to its downward check surface (both
    # 0.525 g in the unit cell) summed over the copies 2 <= |n| <= N
    from paper_1705_02043_gb300 import _binding as b
    p, axis, N = 4, 1, 5
    g = np.array([(-1 + 2 * i / (p - 1), -1 + 2 * j / (p - 1), -1 + 2 * k / (p - 1))
                  for i in range(p) for j in range(p) for k in range(p)
                  if not (0 < i < p - 1 and 0 < j < p - 1 and 0 < k < p - 1)])
    r = 0.525 * (g[:, None, :] - g[None, :, :])
    ref = 0.0
    for n in list(range(-N, -1)) + list(range(2, N + 1)):
        d = r.copy()
        d[..., axis] += n
        rr = np.linalg.norm(d, axis=-1)
        if kernel == 0:
            ref = ref + 1.0 / rr
        else:
            blk = (np.eye(3) / rr[..., None, None] + d[..., :, None] * d[..., None, :] / rr[..., None, None] ** 3)
            ref = ref + (blk / (8 * np.pi)).transpose(0, 2, 1, 3).reshape(len(g) * 3, len(g) * 3)
    M = b.pkifmm_root_operator_finite(kernel, axis, N, p)
    assert np.abs(M - ref).max() <= 1e-13 * np.abs(ref).max()
    assert not np.any(b.pkifmm_root_operator_finite(kernel, axis, 1, p))  # only adjacent copies: no far field


def test_argument_checks_without_a_gpu():
    # the checks that run before any CUDA call: new kernels, finite arrays,
    # periodicity masks
    from paper_1705_02043_gb300 import _binding as b
    lo = (0.0, 0.0, 0.0)
    for args in [(4, 7), (-1, 7)]:  # kernels 0..3 only
        with pytest.raises(pk.PKIFMMError) as e:
            b.pkifmm_plan_create(args[0], args[1], lo, 1.0, 6, 2, 40, 10, 0, 1)
        assert e.value.name == "INVALID_ARG"
    with pytest.raises(pk.PKIFMMError) as e:
        b.pkifmm_plan_create(0, 8, lo, 1.0, 6, 2, 40, 10, 0, 1)  # no such mask
    assert e.value.name == "INVALID_ARG"
    for axis, nimg in [(3, 2), (-1, 2), (0, 0), (1, -4)]:
        with pytest.raises(pk.PKIFMMError) as e:
            b.pkifmm_plan_create_finite(1, axis, nimg, lo, 1.0, 6, 2, 40, 10, 0, 1)
        assert e.value.name == "INVALID_ARG"
    with pytest.raises(pk.PKIFMMError):
        b.pkifmm_root_operator_finite(0, 3, 2, 4)
    with pytest.raises(ValueError):
        pk.PeriodicKIFMM(pk.STOKES, 3, images=2)  # a finite array runs along one axis
