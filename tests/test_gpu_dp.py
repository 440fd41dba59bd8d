"""Doubly periodic (x, y periodic, z free) CUDA path vs the 2D Ewald oracle.

The root operator carries the far images through the closed-form in-plane
mode sums of the library; the oracle takes the k_z integrals by the
trapezoid rule, so agreement checks both.  Tolerances follow the accuracy of
the equivalent surfaces at each p, as for the triply periodic tests."""

import numpy as np
import pytest

import oracle
from gpu_util import rel_l2, run
from paper_1705_02043_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cache(tmp_path_factory):
    return str(tmp_path_factory.mktemp("opcache_dp"))


def _sample(n, k, seed=0):
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


@pytest.mark.parametrize("kernel,p,tol", [(0, 10, 1e-8), (1, 10, 2e-7), (1, 12, 1e-8)])
def test_dp_fp64_gate(kernel, p, tol, cache):
    n = 3000
    if kernel == 0:
        x, q = w.laplace_uniform(n, seed=31)
        d = q[0]
    else:
        x, f = w.stokes_uniform(n, seed=31)
        d = f[0]
    u = run(kernel, 3, x, d, x, p=p, leaf=40, cache_dir=cache)
    ref = oracle.doubly_periodic(kernel, x, d, x)
    e = rel_l2(u, ref)
    print(f"dp fp64 kernel {kernel} p={p} rel_l2 {e:.3e}")
    assert e < tol


def test_dp_error_falls_with_p(cache):
    x, f = w.stokes_uniform(1500, seed=32)
    ref = oracle.stokes_dp(x, f[0], x)
    errs = [rel_l2(run(1, 3, x, f[0], x, p=p, leaf=30, cache_dir=cache), ref) for p in (4, 6, 8)]
    print("stokes DP errors p=4,6,8", errs)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-5


def test_dp_ell_independence(cache):
    x, q = w.laplace_uniform(1200, seed=33)
    us = [run(0, 3, x, q[0], x, p=6, leaf=30, ell=ell, cache_dir=cache) for ell in (1, 2, 3)]
    assert rel_l2(us[1], us[0]) < 1e-11 and rel_l2(us[2], us[0]) < 1e-11


def test_dp_inplane_translation_invariance(cache):
    x, f = w.stokes_uniform(1500, seed=34)
    a = run(1, 3, x, f[0], x, p=8, leaf=30, cache_dir=cache)
    xs = x + np.array([0.37, -0.21, 0.0])
    b = run(1, 3, xs, f[0], xs, p=8, leaf=30, cache_dir=cache)
    assert rel_l2(b, a) < 1e-5


@pytest.mark.parametrize("precision,tol", [(0, 2e-7), (1, 2e-5)])
def test_dp_clustered_slab(precision, tol, cache):
    """Gaussian clusters (sigma 0.02) in the slab z in [0, 0.2], Stokes, p = 10,
    adaptive tree down to depth 12 (the shape of the 4M-point workload)."""
    n = 40000
    x, f = w.clustered_slab(n, seed=35, nclusters=64, sigma=0.02, zlo=0.0, zhi=0.2, kdim=3)
    u = run(1, 3, x, f, x, p=10, leaf=64, depth=12, precision=precision, cache_dir=cache)
    idx = _sample(n, 400)
    ref = oracle.stokes_dp(x, f, x[idx])
    e = rel_l2(u[idx], ref)
    print(f"dp slab precision {precision} rel_l2 {e:.3e}")
    assert e < tol


# doubly periodic in (x, z) and (y, z): the library evaluates the (x, y) case in
# a permuted frame; the oracle is the (x, y) sum on the permuted points
_PERM = {5: [0, 2, 1], 6: [1, 2, 0]}


@pytest.mark.parametrize("kernel,mask", [(0, 5), (0, 6), (1, 5), (1, 6)])
def test_dp_other_axis_pairs(kernel, mask, cache):
    n = 3000
    if kernel == 0:
        x, q = w.laplace_uniform(n, seed=71)
        d = q[0]
    else:
        x, f = w.stokes_uniform(n, seed=71)
        d = f[0]
    u = run(kernel, mask, x, d, x, p=10, leaf=40, cache_dir=cache)
    pm = _PERM[mask]
    ref = oracle.doubly_periodic(kernel, x[:, pm], d[:, pm] if kernel == 1 else d, x[:, pm])
    if kernel == 1:
        back = np.empty_like(ref)
        back[:, pm] = ref  # vector components back to the caller's frame
        ref = back
    e = rel_l2(u, ref)
    print(f"dp mask {mask} kernel {kernel}: rel_l2 {e:.3e}")
    assert e < (1e-8 if kernel == 0 else 2e-7)


def test_dp_other_axis_pairs_pressure_and_field():
    import torch
    import paper_1705_02043_gb300 as pk
    x, f = w.stokes_uniform(2000, seed=72)
    dev = torch.device("cuda:0")
    tx = torch.tensor(x, device=dev)
    plan = pk.PeriodicKIFMM(pk.STOKES_PRESSURE, 5, p=10, leaf_max=40)
    u = plan.evaluate(tx, torch.tensor(f, device=dev), tx).cpu().numpy()[0]
    plan.close()
    pm = _PERM[5]
    idx = np.arange(0, len(x), 37)
    ref_p = oracle.stokes_pressure(3, x[:, pm], f[0][:, pm], x[idx][:, pm])
    assert rel_l2(u[idx, 3], ref_p) < 1e-7
    xq, q = w.laplace_uniform(2000, seed=73)
    plan = pk.PeriodicKIFMM(pk.LAPLACE_FIELD, 6, p=10, leaf_max=40)
    v = plan.evaluate(torch.tensor(xq, device=dev), torch.tensor(q[:, :, None], device=dev),
                      torch.tensor(xq, device=dev)).cpu().numpy()[0]
    plan.close()
    pm = _PERM[6]
    ref = oracle.laplace_field(3, xq[:, pm], q[0], xq[idx][:, pm])
    g = np.empty((len(idx), 3))
    g[:, pm] = ref[:, 1:]
    # measured: potential 2.6e-9, gradient 1.6e-8 (p = 10, 2000 points)
    assert rel_l2(v[idx, 0], ref[:, 0]) < 1e-8 and rel_l2(v[idx, 1:], g) < 5e-8
