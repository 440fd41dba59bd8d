"""A finite array of cells (the finite-length channel of Sec. 4) against the
oracle's plain sum over the copies: the same octree and lists as one periodic
axis, a root operator summed over the non-adjacent copies, no compatibility
condition, no wrapping."""

import numpy as np
import pytest

import oracle
import paper_1705_02043_gb300 as pk
from gpu_util import rel_l2
from paper_1705_02043_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def _eval(kernel, mask, nimg, x, dens, p, precision=0, leaf=40):
    import torch
    k = 1 if kernel == 0 else 3
    plan = pk.PeriodicKIFMM(kernel, mask, p=p, leaf_max=leaf, precision=precision, images=nimg)
    dev = torch.device("cuda:0")
    tx = torch.tensor(x, device=dev)
    out = plan.evaluate(tx, torch.tensor(np.ascontiguousarray(dens.reshape(1, len(x), k)), device=dev), tx)
    torch.cuda.synchronize()
    plan.close()
    u = out.cpu().numpy()[0]
    return u[:, 0] if k == 1 else u


@pytest.mark.parametrize("kernel,mask,nimg", [(0, 1, 3), (0, 2, 20), (0, 4, 1), (1, 4, 4), (1, 1, 12)])
def test_finite_array_fp64(kernel, mask, nimg):
    rng = np.random.default_rng(61 + nimg)
    n = 3000
    x = rng.random((n, 3))
    d = rng.standard_normal(n) if kernel == 0 else rng.standard_normal((n, 3))  # no neutrality needed
    u = _eval(kernel, mask, nimg, x, d, p=10)
    idx = np.arange(0, n, 31)
    ref = oracle.finite_array(kernel, {1: 0, 2: 1, 4: 2}[mask], nimg, x, d, x[idx])
    e = rel_l2(u[idx], ref)
    print(f"finite array kernel {kernel} axis mask {mask} N={nimg}: rel_l2 {e:.2e}")
    assert e < 1e-7  # measured 3e-10..3e-8 at p = 10


def test_finite_array_mixed():
    x, f = w.stokes_uniform(20000, seed=62)
    u = _eval(1, 2, 10, x, f[0], p=8, precision=pk.MIXED, leaf=64)
    idx = np.arange(0, len(x), 401)
    e = rel_l2(u[idx], oracle.finite_array(1, 1, 10, x, f[0], x[idx]))
    print(f"finite array mixed: rel_l2 {e:.2e}")
    assert e < 2e-5  # measured 5.4e-6


def test_finite_array_points_stay_in_the_cell():
    rng = np.random.default_rng(63)
    x = rng.random((200, 3))
    x[7, 0] = 1.25  # along the array axis: not wrapped, rejected
    with pytest.raises(pk.PKIFMMError) as e:
        _eval(0, 1, 3, x, rng.standard_normal(200), p=6)
    assert e.value.code == -2
