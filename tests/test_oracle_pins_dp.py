"""Pins of the doubly periodic (x, y periodic, z free) oracle.

The doubly periodic Ewald sum is not written out in the paper (Sec. 3.3
refers to the literature for it), so the oracle's 2D split is checked
against facts that do not depend on how it is split:

* independence of the splitting parameter xi;
* brute-force in-plane image sums for cells whose force (charge) moments of
  order 0, 1 and 2 vanish (eight cube vertices with alternating signs), where
  the 2D lattice sum converges absolutely;
* the plane average of the field: the k_par = 0 part of the full kernel is
  the field of a uniform sheet, so over any plane z = z0 clear of the points
  the mean of u_z is 0 (zero net flux, Sec. 3.3) and the mean of the in-plane
  velocity is -(1/2A) sum_s f_s |z0 - z_s| (Laplace: -(2 pi/A) sum_s q_s |z0 - z_s|);
* the far-field limits: u tends to +-(1/2A) sum_s f_s z_s as z -> +-inf
  (Laplace: +-(2 pi/A) sum_s q_s z_s).
"""

import numpy as np
import pytest

import oracle


def _neutral_slab(n, seed, z0=0.3, z1=0.7):
    rng = np.random.default_rng(seed)
    y = rng.random((n, 3))
    y[:, 2] = z0 + (z1 - z0) * y[:, 2]
    q = rng.uniform(-1, 1, n)
    q -= q.mean()
    f = rng.standard_normal((n, 3))
    f -= f.mean(0)
    return y, q, f


def _octupole_cell(c, d):
    y, s = [], []
    for i in (0, 1):
        for j in (0, 1):
            for k in (0, 1):
                sg = np.array([2 * i - 1, 2 * j - 1, 2 * k - 1])
                y.append(c + d * sg)
                s.append(float(sg.prod()))
    return np.array(y), np.array(s)


def _image_sum(kernel, y, dens, x, M):
    """Plain sum over the in-plane images |n|_inf <= M."""
    n = np.arange(-M, M + 1)
    nx, ny = np.meshgrid(n, n, indexing="ij")
    sh = np.stack([nx.ravel(), ny.ravel(), np.zeros(nx.size)], 1)
    out = np.zeros((len(x), 1 if kernel == 0 else 3))
    for t in range(len(x)):
        for s in range(len(y)):
            d = x[t] - y[s] - sh
            r2 = np.einsum("ij,ij->i", d, d)
            r = np.sqrt(r2)
            if kernel == 0:
                out[t, 0] += np.sum(dens[s] / r)
            else:
                df = d @ dens[s]
                out[t] += (dens[s] * np.sum(1 / r) + (d * (df / (r2 * r))[:, None]).sum(0)) / (8 * np.pi)
    return out[:, 0] if kernel == 0 else out


@pytest.mark.parametrize("kernel", [0, 1])
def test_dp_xi_independence(kernel):
    y, q, f = _neutral_slab(60, 1)
    d = q if kernel == 0 else f
    x = np.random.default_rng(2).random((12, 3))
    x[:, 2] = -0.2 + 1.4 * x[:, 2]
    us = [oracle.doubly_periodic(kernel, y, d, x, rc=rc) for rc in (0.75, 1.0, 1.4)]
    scale = np.abs(us[1]).max()
    assert np.abs(us[0] - us[1]).max() < 1e-13 * scale
    assert np.abs(us[2] - us[1]).max() < 1e-13 * scale


def test_dp_brute_force_octupole_cells():
    y, s = _octupole_cell(np.array([0.4, 0.55, 0.5]), 0.1)
    f = s[:, None] * np.array([0.3, -0.7, 0.5])[None, :]
    x = np.array([[0.1, 0.2, 0.3], [0.9, 0.5, 0.75], [0.45, 0.5, 0.1], [0.3, 0.8, 1.4]])
    ref = oracle.laplace_dp(y, s, x)
    b = _image_sum(0, y, s, x, 100)
    assert np.abs(b - ref).max() < 1e-10 * np.abs(ref).max()
    ref = oracle.stokes_dp(y, f, x)
    b1, b2 = _image_sum(1, y, f, x, 100), _image_sum(1, y, f, x, 200)
    # the truncation error falls like M^-3: one Richardson step
    rich = (8 * b2 - b1) / 7
    assert np.abs(b2 - ref).max() < 1e-8 * np.abs(ref).max()
    assert np.abs(rich - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("rc", [1.0, 1.5])
def test_dp_plane_mean_is_sheet_field(rc):
    y, q, f = _neutral_slab(30, 3)
    g = (np.arange(48) + 0.5) / 48
    gx, gy = np.meshgrid(g, g, indexing="ij")
    for z0 in (0.05, 0.95):
        x = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, z0)], 1)
        u = oracle.stokes_dp(y, f, x, rc=rc)
        scale = np.abs(u).max()
        assert abs(u[:, 2].mean()) < 1e-12 * scale  # zero net flux through the plane
        sheet = -0.5 * (f[:, :2] * np.abs(z0 - y[:, 2])[:, None]).sum(0)
        assert np.abs(u[:, :2].mean(0) - sheet).max() < 1e-12 * scale
        phi = oracle.laplace_dp(y, q, x, rc=rc)
        sheet = -2 * np.pi * np.sum(q * np.abs(z0 - y[:, 2]))
        assert abs(phi.mean() - sheet) < 1e-12 * np.abs(phi).max()


def test_dp_far_field_limits():
    y, q, f = _neutral_slab(40, 4)
    x = np.array([[0.2, 0.7, 4.7], [0.6, 0.1, 4.7], [0.2, 0.7, -3.7], [0.9, 0.4, -3.7]])
    u = oracle.stokes_dp(y, f, x)
    lim = 0.5 * (f[:, :2] * y[:, 2:3]).sum(0)
    scale = np.abs(lim).max()
    for t, sgn in enumerate((1, 1, -1, -1)):
        assert np.abs(u[t, :2] - sgn * lim).max() < 1e-9 * scale
        assert abs(u[t, 2]) < 1e-9 * scale
    phi = oracle.laplace_dp(y, q, x)
    lim = 2 * np.pi * np.sum(q * y[:, 2])
    for t, sgn in enumerate((1, 1, -1, -1)):
        assert abs(phi[t] - sgn * lim) < 1e-9 * abs(lim)
