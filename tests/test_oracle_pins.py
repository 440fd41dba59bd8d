"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the paper's
worked example, classical lattice constants, closed-form series, brute-force
lattice sums that converge absolutely, splitting-parameter independence and
physical invariants (Stokes' law, zero net flux).
"""

import math
import os

import numpy as np
import pytest

import oracle
from paper_1705_02043_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Classical constants (not from the paper): simple-cubic lattice with a
# neutralising background, potential at a unit charge from its images
# (Wigner / Hasimoto constant), and the NaCl Madelung constant.
SC_CONSTANT = 2.837297479480620
NACL_MADELUNG = 1.747564594633182


def _golden_madelung():
    src, q, trg, exact = [], [], [], None
    for line in open(os.path.join(GOLDEN, "madelung_1d.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "source":
            src.append([float(v) for v in f[1:4]]); q.append(float(f[4]))
        elif f[0] == "target":
            trg.append([float(v) for v in f[1:4]])
        elif f[0] == "exact":
            exact = float(f[1])
    return np.array(src), np.array(q), np.array(trg), exact


# ---------------- singly periodic Laplace ----------------

def test_madelung_1d_paper_example():
    """Sec. 3.2 worked example: -8 ln 2 at both positive charges."""
    src, q, trg, exact = _golden_madelung()
    assert exact == pytest.approx(-8 * math.log(2), abs=1e-15)
    v = oracle.laplace_sp(src, q, trg, axis=2)
    assert np.max(np.abs(v - exact)) < 1e-13
    # the same chain along x and along y (axis handling, box length L)
    for axis in (0, 1):
        perm = [2, 0, 1] if axis == 0 else [0, 2, 1]
        v = oracle.laplace_sp(src[:, perm] * 3.0, q, trg[:, perm] * 3.0, axis=axis, L=3.0)
        assert np.max(np.abs(v - exact / 3.0)) < 1e-13


def _k0_series_potential(x_rel, rho, terms=40):
    """Unit-period 1D lattice sum of 1/r as a Bessel series, up to a constant:
    -2 ln rho + 4 sum_k K0(2 pi k rho) cos(2 pi k x)."""
    from scipy.special import k0
    k = np.arange(1, terms + 1)
    return -2 * np.log(rho) + 4 * np.sum(k0(2 * np.pi * k * rho) * np.cos(2 * np.pi * k * x_rel))


def test_sp_matches_bessel_series():
    """Independent formula: for rho >= 0.1 the K0 series converges fast."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        y1, y2, x = rng.random(3), rng.random(3), rng.random(3)
        r1, r2 = x - y1, x - y2
        rho1, rho2 = np.hypot(r1[1], r1[2]), np.hypot(r2[1], r2[2])
        if min(rho1, rho2) < 0.1:
            continue
        ref = _k0_series_potential(r1[0], rho1) - _k0_series_potential(r2[0], rho2)
        v = oracle.laplace_sp(np.array([y1, y2]), np.array([1.0, -1.0]), x[None], axis=0)[0]
        assert v == pytest.approx(ref, abs=1e-13)


def test_sp_brute_force_converges_like_inverse_square():
    """Neutral direct image sums converge like 1/M^2 (Sec. 3.2) to the oracle."""
    x, q = w.laplace_sp_uniform(12, seed=3)
    trg = x[:4]
    ref = oracle.laplace_sp(x, q, trg, axis=0)

    def brute(M):
        out = np.zeros(len(trg))
        for n in range(-M, M + 1):
            d = trg[:, None, :] - (x[None, :, :] + np.array([n, 0, 0]))
            r = np.linalg.norm(d, axis=-1)
            with np.errstate(divide="ignore"):
                out += np.where(r > 0, q[None, :] / r, 0.0).sum(1)
        return out

    e1, e2 = np.abs(brute(200) - ref).max(), np.abs(brute(400) - ref).max()
    assert e2 < 1e-4 and 3.0 < e1 / e2 < 5.0  # second-order convergence


def test_sp_periodicity_and_translation():
    x, q = w.laplace_sp_uniform(50, seed=4)
    trg = w.uniform_points(5, seed=40)
    a = oracle.laplace_sp(x, q, trg, axis=1)
    b = oracle.laplace_sp(x, q, trg + np.array([0, 1.0, 0]), axis=1)
    c = oracle.laplace_sp(x + 0.3, q, trg + 0.3, axis=1)
    assert np.allclose(a, b, atol=1e-13) and np.allclose(a, c, atol=1e-12)


# ---------------- triply periodic Laplace ----------------

def test_tp_laplace_sc_constant_with_background():
    """One charge + neutralising background: -2.837297/L at the charge."""
    for L in (1.0, 2.5):
        y = np.array([[0.3, 0.4, 0.5]]) * L
        v = oracle.laplace_tp(y, np.array([1.0]), y, L=L)
        assert v[0] == pytest.approx(-SC_CONSTANT / L, abs=1e-12)


def test_tp_laplace_nacl_madelung():
    """Rock salt: 8 alternating ions at spacing L/2, potential -M/(L/2) at a + ion."""
    pts = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)]) * 0.5 + 0.1
    q = np.array([(-1.0) ** (i + j + k) for i in range(2) for j in range(2) for k in range(2)])
    v = oracle.laplace_tp(pts, q, pts)
    assert np.allclose(v * q, -2 * NACL_MADELUNG, atol=1e-12)


def test_tp_laplace_xi_independence():
    x, q = w.laplace_uniform(40, seed=7)
    q = q[0]
    ref = oracle.laplace_tp(x, q, x, xi=6.0, rc=1.0)
    for xi in (4.0, 8.0, 12.0):
        v = oracle.laplace_tp(x, q, x, xi=xi)
        assert np.max(np.abs(v - ref)) < 1e-12 * np.max(np.abs(ref))


def _octupole_cell(center, d, sign=1.0):
    o = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)], float)
    q = np.array([(-1.0) ** (i + j + k) for i in range(2) for j in range(2) for k in range(2)])
    return center + d * (o - 0.5), sign * q


def _cube_lattice_sum(y, dens, x, R, stokes):
    """sum over images |n|_inf <= R, skipping coincident pairs (numpy brute force)."""
    n = np.arange(-R, R + 1, dtype=float)
    img = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3)
    out = np.zeros((len(x), 3 if stokes else 1))
    for s in range(len(y)):
        d = x[:, None, :] - (y[s] + img)[None]  # [T, I, 3]
        r2 = (d * d).sum(-1)
        ok = r2 > 0
        r = np.sqrt(np.where(ok, r2, 1.0))
        if not stokes:
            out[:, 0] += np.where(ok, dens[s] / r, 0.0).sum(1)
        else:
            f = dens[s]
            df = (d * f).sum(-1)
            u = (f[None, None, :] / r[..., None] + d * (df / r ** 3)[..., None]) / (8 * np.pi)
            out += np.where(ok[..., None], u, 0.0).sum(1)
    return out


def test_tp_laplace_brute_force_octupole_cell():
    """Cells with vanishing charge, dipole and second moments: cube-ordered
    lattice sums converge absolutely to the Ewald value."""
    y, q = _octupole_cell(np.array([0.42, 0.55, 0.37]), 0.2)
    x = np.array([[0.1, 0.2, 0.3], [0.8, 0.7, 0.9], y[0]])
    ref = oracle.laplace_tp(y, q, x)
    b1 = _cube_lattice_sum(y, q, x, 12, False)[:, 0]
    b2 = _cube_lattice_sum(y, q, x, 24, False)[:, 0]
    e1, e2 = np.max(np.abs(b1 - ref)), np.max(np.abs(b2 - ref))
    assert e2 < 1e-8 and e2 < 0.5 * e1


# ---------------- triply periodic Stokes ----------------

def test_tp_stokes_hasimoto_self_constant():
    """Single force, zero mean flow: the images move it by -2.837297 f/(6 pi L)."""
    y, f = w.single_force()
    for L in (1.0, 3.0):
        u = oracle.stokes_tp(y * L, f, y * L, L=L)
        assert np.allclose(u, -SC_CONSTANT / (6 * np.pi * L) * f, atol=1e-13)


def test_tp_stokes_xi_independence():
    x, f = w.stokes_uniform(30, seed=2, neutral=False)
    f = f[0]
    ref = oracle.stokes_tp(x, f, x, xi=6.0, rc=1.0)
    for xi in (4.0, 9.0, 14.0):
        v = oracle.stokes_tp(x, f, x, xi=xi)
        assert np.max(np.abs(v - ref)) < 1e-12 * np.max(np.abs(ref))


def test_tp_stokes_brute_force_zero_moment_cell():
    y, s = _octupole_cell(np.array([0.33, 0.61, 0.47]), 0.2)
    fdir = np.array([0.3, -1.0, 0.6])
    f = s[:, None] * fdir[None, :]
    x = np.array([[0.1, 0.2, 0.3], [0.75, 0.05, 0.9]])
    ref = oracle.stokes_tp(y, f, x)
    b1 = _cube_lattice_sum(y, f, x, 12, True)
    b2 = _cube_lattice_sum(y, f, x, 24, True)
    # the truncation error is c/R^2 here (cubic symmetry cancels the slower
    # shell terms), so one Richardson step removes it
    rich = (4 * b2 - b1) / 3
    assert np.max(np.abs(b2 - ref)) < 1e-6
    assert np.max(np.abs(rich - ref)) < 1e-7


def _clenshaw_curtis_01(m):
    """Clenshaw-Curtis nodes (1-cos(pi i/(m-1)))/2 and weights on [0,1]."""
    n = m - 1
    theta = np.pi * np.arange(m) / n
    wts = np.zeros(m)
    for i in range(m):
        s = 0.0
        for k in range(1, n // 2 + 1):
            b = 1.0 if 2 * k == n else 2.0
            s += b / (4 * k * k - 1) * np.cos(2 * k * theta[i])
        c = 1.0 if i in (0, n) else 2.0
        wts[i] = c / n * (1 - s)
    return 0.5 * (1 - np.cos(theta)), 0.5 * wts


def test_tp_stokes_zero_net_flux_on_faces():
    """Sec. 3.4: zero mean flow makes the flux through each face vanish."""
    y, f = w.single_force()
    y2, f2 = w.two_forces()
    c, wt = _clenshaw_curtis_01(49)
    assert abs(wt.sum() - 1) < 1e-14
    A, B = np.meshgrid(c, c, indexing="ij")
    W2 = np.outer(wt, wt).ravel()
    for ys, fs in ((y, f), (y2, f2)):
        for axis in range(3):
            face = np.zeros((c.size ** 2, 3))
            others = [a for a in range(3) if a != axis]
            face[:, others[0]], face[:, others[1]] = A.ravel(), B.ravel()
            u = oracle.stokes_tp(ys, fs, face)
            flux = np.sum(W2 * u[:, axis])
            assert abs(flux) < 1e-11 * np.max(np.abs(u))


# ---------------- free space ----------------

def test_stokeslet_sphere_average_is_stokes_law():
    """Mean velocity on a sphere of radius a around a point force: f/(6 pi a)."""
    rng = np.random.default_rng(0)
    f = rng.standard_normal(3)
    # the octahedron vertices and the cube vertices are spherical 3-designs:
    # exact for the degree-2 polynomial (I + r r^T)/a on the sphere
    a = 0.37
    octa = np.concatenate([np.eye(3), -np.eye(3)])
    cube = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)]) / np.sqrt(3)
    pts = a * np.concatenate([octa, cube]) + 0.5
    u = oracle.free_space(oracle.STOKES, np.array([[0.5, 0.5, 0.5]]), f[None], pts)
    assert np.allclose(u[:6].mean(0), f / (6 * np.pi * a), rtol=1e-14)
    assert np.allclose(u[6:].mean(0), f / (6 * np.pi * a), rtol=1e-14)
    ql = oracle.free_space(oracle.LAPLACE, np.array([[0.5, 0.5, 0.5]]), np.array([2.0]), pts)
    assert np.allclose(ql, 2.0 / a, rtol=1e-14)


def test_stokeslet_solves_stokes_equations():
    """Finite differences: div u = 0 and -lap u + grad p = 0 away from the force,
    with pressure p = f.r/(4 pi r^3)."""
    f = np.array([0.3, -0.7, 1.1])
    y = np.zeros((1, 3))
    x0 = np.array([0.31, -0.22, 0.17])
    h = 1e-3
    E = np.eye(3)

    def u(x):
        return oracle.free_space(oracle.STOKES, y, f[None], np.atleast_2d(x))[0]

    def p(x):
        return f @ x / (4 * np.pi * np.linalg.norm(x) ** 3)

    div = sum((u(x0 + h * E[a])[a] - u(x0 - h * E[a])[a]) / (2 * h) for a in range(3))
    lap = sum((u(x0 + h * E[a]) - 2 * u(x0) + u(x0 - h * E[a])) / h ** 2 for a in range(3))
    gp = np.array([(p(x0 + h * E[a]) - p(x0 - h * E[a])) / (2 * h) for a in range(3)])
    assert abs(div) < 1e-5
    assert np.max(np.abs(-lap + gp)) < 1e-4


def test_error_metrics_definitions():
    u = np.array([[1.0, 2.0], [3.0, 4.0]])
    ref = np.array([[1.0, 2.5], [3.0, 3.0]])
    m = oracle.error_metrics(u, ref)
    assert m["max_abs"] == 1.0 and m["mean_abs"] == 0.375
    assert m["rms"] == pytest.approx(math.sqrt(1.25 / 4))
    assert m["rel_l2"] == pytest.approx(math.sqrt(1.25) / math.sqrt(1 + 6.25 + 9 + 9))


def test_stokes_tp_hasimoto_matches_beenakker_split():
    """Two splits of the same triply periodic Stokes sum (Hasimoto's Fourier
    weight (1 + a) e^{-a}, Beenakker's (1 + a + 2a^2) e^{-a}, a = k^2/4xi^2,
    each with its own real-space kernel and self term) give the same
    velocities, with and without a net force."""
    rng = np.random.default_rng(31)
    y = rng.random((60, 3))
    x = rng.random((8, 3))
    for neutral in (False, True):
        f = rng.standard_normal((60, 3))
        if neutral:
            f -= f.mean(0)
        h = oracle.stokes_tp(y, f, x)
        for rc in (0.8, 1.2):
            b = oracle.stokes_tp_beenakker(y, f, x, rc=rc)
            assert np.abs(b - h).max() < 1e-13 * np.abs(h).max()
