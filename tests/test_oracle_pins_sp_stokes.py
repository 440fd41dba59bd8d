"""Pins of the singly periodic Stokes oracle.

For zero net force the symmetric image sum converges (the 1/n monopole
terms cancel between sources, the dipole terms between the images +n and
-n), with a truncation error falling like M^-2.  The oracle instead sums each
pair with a pair-independent 1/n regularisation and a closed-form
Euler-Maclaurin tail, so the plain sum, extrapolated in M, is an independent
check of both the regularisation and the tail."""

import numpy as np
import pytest

import oracle


def _neutral(n, seed):
    rng = np.random.default_rng(seed)
    y = rng.random((n, 3))
    f = rng.standard_normal((n, 3))
    f -= f.mean(0)
    return y, f


def _plain(y, f, x, axis, M):
    n = np.arange(-M, M + 1)
    out = np.zeros((len(x), 3))
    for t in range(len(x)):
        for s in range(len(y)):
            r = x[t] - y[s]
            r[axis] -= np.floor(r[axis] + 0.5)
            d = np.tile(r, (len(n), 1))
            d[:, axis] += n
            r2 = np.einsum("ij,ij->i", d, d)
            rr = np.sqrt(r2)
            out[t] += (f[s] * np.sum(1 / rr) + (d * ((d @ f[s]) / (r2 * rr))[:, None]).sum(0)) / (8 * np.pi)
    return out


@pytest.mark.parametrize("axis", [0, 2])
def test_stokes_sp_matches_plain_sum_extrapolated(axis):
    y, f = _neutral(12, 1 + axis)
    x = np.random.default_rng(9).random((4, 3))
    ref = oracle.stokes_sp(y, f, x, axis=axis)
    b1, b2 = _plain(y, f, x, axis, 1500), _plain(y, f, x, axis, 3000)
    scale = np.abs(ref).max()
    assert np.abs(b2 - ref).max() < 1e-7 * scale          # plain sum, error ~ M^-2
    assert np.abs((4 * b2 - b1) / 3 - ref).max() < 1e-10 * scale


def test_stokes_sp_independent_of_truncation():
    y, f = _neutral(15, 3)
    x = np.random.default_rng(4).random((5, 3))
    # the three-term Euler-Maclaurin tail leaves an error ~ M^-6: 2e-13 at M = 80
    a, b = oracle.stokes_sp(y, f, x, M=80), oracle.stokes_sp(y, f, x, M=2000)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_stokes_sp_periodic_and_symmetric():
    y, f = _neutral(10, 5)
    x = np.random.default_rng(6).random((3, 3))
    u = oracle.stokes_sp(y, f, x, axis=1)
    xs = x.copy()
    xs[:, 1] += 1.0
    assert np.abs(oracle.stokes_sp(y, f, xs, axis=1) - u).max() < 1e-13 * np.abs(u).max()
    # reflection z -> -z of every point flips the z component only (the kernel is even)
    yr, xr, fr = y * [1, 1, -1], x * [1, 1, -1], f * [1, 1, -1]
    ur = oracle.stokes_sp(yr, fr, xr, axis=1)
    assert np.abs(ur - u * [1, 1, -1]).max() < 1e-13 * np.abs(u).max()
