"""Pins of the oracle's Laplace field (potential gradient) and Stokes pressure.

The gradient sums are checked against Richardson-extrapolated central
differences of the potential oracle (pinned on its own in
test_oracle_pins*.py), against their own splitting parameters, and the
pressure against the free-space formula p = f.r/(4 pi r^3) and against the
Stokes equations grad p = lap u (mu = 1, away from the sources), with u the
independently pinned velocity oracle."""

import numpy as np
import pytest

import oracle

PERIODIC = [0, 7, 3, 1, 2, 4]


def _charges(n, seed):
    rng = np.random.default_rng(seed)
    y = rng.random((n, 3))
    q = rng.standard_normal(n)
    return y, q - q.mean()


def _richardson_gradient(fun, xt, h=1e-4):
    g = np.zeros((len(xt), 3))
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        d1 = (fun(xt + e) - fun(xt - e)) / (2 * h)
        d2 = (fun(xt + 2 * e) - fun(xt - 2 * e)) / (4 * h)
        g[:, c] = (4 * d1 - d2) / 3
    return g


@pytest.mark.parametrize("periodic", PERIODIC)
def test_gradient_matches_differences_of_the_potential(periodic):
    y, q = _charges(40, 3)
    xt = np.random.default_rng(4).random((6, 3)) * 0.9 + 0.05
    g = oracle.laplace_gradient(periodic, y, q, xt)
    fd = _richardson_gradient(lambda X: oracle.periodic_sum(oracle.LAPLACE, periodic, y, q, X), xt)
    assert np.abs(g - fd).max() <= 1e-8 * np.abs(g).max()


def test_gradient_independent_of_splitting():
    y, q = _charges(30, 5)
    xt = np.random.default_rng(6).random((5, 3))
    for periodic in (7, 3):
        a = oracle.laplace_gradient(periodic, y, q, xt, xi=5.0)
        b = oracle.laplace_gradient(periodic, y, q, xt, xi=9.0)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    a = oracle.laplace_gradient(1, y, q, xt, M=60)
    b = oracle.laplace_gradient(1, y, q, xt, M=400)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_gradient_scales_with_the_box():
    # K = 1/r is homogeneous of degree -1: the field of the scaled problem is 1/L^2 times
    y, q = _charges(20, 7)
    xt = np.random.default_rng(8).random((4, 3))
    L = 2.5
    for periodic in (7, 3, 4):
        a = oracle.laplace_gradient(periodic, y, q, xt)
        b = oracle.laplace_gradient(periodic, L * y, q, L * xt, L=L)
        assert np.abs(a / L ** 2 - b).max() <= 1e-12 * np.abs(b).max()


def test_pressure_free_space_formula():
    rng = np.random.default_rng(9)
    y, f = rng.random((25, 3)), rng.standard_normal((25, 3))
    xt = rng.random((7, 3))
    d = xt[:, None, :] - y[None, :, :]
    r = np.linalg.norm(d, axis=2)
    ref = ((d * f[None]).sum(2) / (4 * np.pi * r ** 3)).sum(1)
    assert np.abs(oracle.stokes_pressure(0, y, f, xt) - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("periodic", [0, 7, 3, 1, 4])
def test_pressure_satisfies_the_stokes_equations(periodic):
    # grad p = lap u away from the sources (mu = 1), fourth-order stencils
    rng = np.random.default_rng(11)
    y, f = rng.random((30, 3)), rng.standard_normal((30, 3))
    f -= f.mean(0)
    xt = np.array([[0.31, 0.47, 0.52], [0.8, 0.15, 0.66]])
    h = 2e-3
    u = lambda X: oracle.periodic_sum(oracle.STOKES, periodic, y, f, X)
    p = lambda X: oracle.stokes_pressure(periodic, y, f, X)
    gp, lap = np.zeros((2, 3)), np.zeros((2, 3))
    u0 = u(xt)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        gp[:, c] = (8 * (p(xt + e) - p(xt - e)) - (p(xt + 2 * e) - p(xt - 2 * e))) / (12 * h)
        lap += (-u(xt + 2 * e) + 16 * u(xt + e) - 30 * u0 + 16 * u(xt - e) - u(xt - 2 * e)) / (12 * h * h)
    assert np.abs(gp - lap).max() <= 1e-6 * np.abs(gp).max()
