"""Pins of the oracle's finite array of cells (the finite-length channel of
Sec. 4): no images equals free space; the array converges to the singly
periodic sum (pinned on its own) as the image count grows, at the rate its
neutral tail fixes; the sum is symmetric under the mirror image of the array."""

import numpy as np

import oracle


def _charges(n, seed):
    rng = np.random.default_rng(seed)
    y = rng.random((n, 3))
    q = rng.standard_normal(n)
    return y, q - q.mean()


def test_no_images_is_free_space():
    y, q = _charges(50, 1)
    xt = np.random.default_rng(2).random((7, 3))
    np.testing.assert_array_equal(oracle.finite_array(0, 0, 0, y, q, xt), oracle.free_space(0, y, q, xt))


def test_converges_to_the_singly_periodic_sum():
    # neutral charges: the tail of the image sum beyond N falls like 1/N^2
    # (dipole images), so doubling N divides the gap by about 4
    y, q = _charges(40, 3)
    xt = np.random.default_rng(4).random((5, 3))
    sp = oracle.laplace_sp(y, q, xt, axis=1, M=2000)
    gaps = [np.abs(oracle.finite_array(0, 1, n, y, q, xt) - sp).max() for n in (100, 200, 400)]
    assert gaps[2] < 1e-4 * np.abs(sp).max()
    assert 3.0 < gaps[0] / gaps[1] < 5.0 and 3.0 < gaps[1] / gaps[2] < 5.0


def test_stokes_converges_to_the_singly_periodic_sum():
    rng = np.random.default_rng(5)
    y, f = rng.random((30, 3)), rng.standard_normal((30, 3))
    f -= f.mean(0)
    xt = rng.random((4, 3))
    sp = oracle.stokes_sp(y, f, xt, 2)
    gaps = [np.abs(oracle.finite_array(1, 2, n, y, f, xt) - sp).max() for n in (100, 200)]
    assert gaps[1] < 1e-4 * np.abs(sp).max() and 3.0 < gaps[0] / gaps[1] < 5.0


def test_mirror_symmetry():
    # reflecting sources and targets through the cell's mid-plane normal to the
    # axis maps the array onto itself: Laplace potentials are unchanged
    y, q = _charges(30, 6)
    xt = np.random.default_rng(7).random((6, 3))
    a = oracle.finite_array(0, 0, 5, y, q, xt)
    ym, xm = y.copy(), xt.copy()
    ym[:, 0] = 1.0 - ym[:, 0]
    xm[:, 0] = 1.0 - xm[:, 0]
    b = oracle.finite_array(0, 0, 5, ym, q, xm)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())
