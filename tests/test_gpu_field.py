"""Laplace field (potential and gradient at the targets) and Stokes velocity
with pressure, CUDA path against the oracle.

Both reuse the Laplace / Stokes translations; only the target evaluations
(L2T, W list, U list, step d) differ, and the pressure is the divergence of
the Laplace fields of the three force components.  Tolerances follow the
surface accuracy at each p; measured, the gradient is as accurate as the
potential (p = 10: both ~3e-9 in TP; p = 6: ~8e-6)."""

import numpy as np
import pytest

import oracle
import paper_1705_02043_gb300 as pk
from gpu_util import rel_l2
from paper_1705_02043_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def _plan_eval(kernel, periodic, x, dens, p, precision=0, leaf=40, nrhs=1, far=None):
    import torch
    plan = pk.PeriodicKIFMM(kernel, periodic, p=p, leaf_max=leaf, precision=precision, nrhs=nrhs)
    if far is not None:
        plan.set_far_field(far)
    dev = torch.device("cuda:0")
    tx = torch.tensor(x, device=dev)
    td = torch.tensor(np.ascontiguousarray(dens.reshape(nrhs, len(x), -1)), device=dev)
    out = plan.evaluate(tx, td, tx)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    plan.close()
    return res


def _points(n, periodic, seed):
    x, q = w.laplace_uniform(n, seed=seed)
    if periodic != 7:
        x = np.clip(x, 0.0, np.nextafter(1.0, 0.0))
    return x, q[0]


@pytest.mark.parametrize("periodic,p,tol_phi,tol_grad", [(7, 10, 2e-8, 2e-8), (3, 10, 2e-8, 2e-8),
                                                         (4, 10, 2e-8, 2e-8), (0, 10, 2e-8, 2e-8),
                                                         (7, 6, 3e-5, 3e-5)])
def test_laplace_field_fp64(periodic, p, tol_phi, tol_grad):
    x, q = _points(3000, periodic, 51)
    u = _plan_eval(pk.LAPLACE_FIELD, periodic, x, q, p)[0]
    idx = np.arange(0, len(x), 29)
    ref = oracle.laplace_field(periodic, x, q, x[idx])
    e_phi, e_grad = rel_l2(u[idx, 0], ref[:, 0]), rel_l2(u[idx, 1:], ref[:, 1:])
    print(f"field periodic {periodic} p={p}: potential {e_phi:.2e}, gradient {e_grad:.2e}")
    assert e_phi < tol_phi and e_grad < tol_grad


def test_laplace_field_potential_is_the_laplace_result():
    x, q = _points(2000, 7, 52)
    u = _plan_eval(pk.LAPLACE_FIELD, 7, x, q, 8)[0]
    v = _plan_eval(pk.LAPLACE, 7, x, q, 8)[0, :, 0]
    assert np.abs(u[:, 0] - v).max() <= 1e-13 * np.abs(v).max()


@pytest.mark.parametrize("periodic", [7, 1])
def test_laplace_field_mixed(periodic):
    x, q = _points(20000, periodic, 53)
    u = _plan_eval(pk.LAPLACE_FIELD, periodic, x, q, 6, precision=pk.MIXED, leaf=64)[0]
    idx = np.arange(0, len(x), 397)
    ref = oracle.laplace_field(periodic, x, q, x[idx])
    e_phi, e_grad = rel_l2(u[idx, 0], ref[:, 0]), rel_l2(u[idx, 1:], ref[:, 1:])
    print(f"field mixed periodic {periodic}: potential {e_phi:.2e}, gradient {e_grad:.2e}")
    assert e_phi < 3e-5 and e_grad < 3e-5


def test_laplace_field_step_d_matches_l2l():
    # Algorithm 2 step d with the field kernel: the two far-field routes agree
    # to the method's error and both meet the oracle
    x, q = _points(2000, 7, 54)
    a = _plan_eval(pk.LAPLACE_FIELD, 7, x, q, 8, far=pk.FAR_L2L)[0]
    b = _plan_eval(pk.LAPLACE_FIELD, 7, x, q, 8, far=pk.FAR_DIRECT)[0]
    ref = oracle.laplace_field(7, x, q, x)
    assert rel_l2(b[:, 0], a[:, 0]) < 1e-6 and rel_l2(b[:, 1:], a[:, 1:]) < 1e-5
    for c in (slice(0, 1), slice(1, 4)):
        assert rel_l2(b[:, c], ref[:, c]) < 3 * max(rel_l2(a[:, c], ref[:, c]), 1e-7)


@pytest.mark.parametrize("periodic,p,tol_u,tol_p", [(7, 10, 5e-7, 5e-8), (3, 10, 5e-7, 5e-8), (1, 10, 5e-7, 5e-8),
                                                    (0, 10, 5e-7, 5e-8)])
def test_stokes_pressure_fp64(periodic, p, tol_u, tol_p):
    x, f = w.stokes_uniform(2000, seed=55)
    f = f[0]
    if periodic != 7:
        x = np.clip(x, 0.0, np.nextafter(1.0, 0.0))
    u = _plan_eval(pk.STOKES_PRESSURE, periodic, x, f, p)[0]
    idx = np.arange(0, len(x), 23)
    ref_u = oracle.periodic_sum(oracle.STOKES, periodic, x, f, x[idx])
    ref_p = oracle.stokes_pressure(periodic, x, f, x[idx])
    e_u, e_p = rel_l2(u[idx, :3], ref_u), rel_l2(u[idx, 3], ref_p)
    print(f"stokes pressure periodic {periodic} p={p}: velocity {e_u:.2e}, pressure {e_p:.2e}")
    assert e_u < tol_u and e_p < tol_p
    v = _plan_eval(pk.STOKES, periodic, x, f, p)[0]
    assert np.abs(u[:, :3] - v).max() <= 1e-13 * np.abs(v).max()


def test_stokes_pressure_mixed_two_vectors():
    x, f = w.stokes_uniform(20000, nrhs=2, seed=56)
    u = _plan_eval(pk.STOKES_PRESSURE, 7, x, f, 8, precision=pk.MIXED, leaf=64, nrhs=2)
    idx = np.arange(0, len(x), 401)
    for r in range(2):
        ref_p = oracle.stokes_pressure(7, x, f[r], x[idx])
        ref_u = oracle.periodic_sum(oracle.STOKES, 7, x, f[r], x[idx])
        e_u, e_p = rel_l2(u[r, idx, :3], ref_u), rel_l2(u[r, idx, 3], ref_p)
        print(f"stokes pressure mixed vector {r}: velocity {e_u:.2e}, pressure {e_p:.2e}")
        assert e_u < 3e-5 and e_p < 2e-5


def test_stokes_pressure_needs_zero_net_force():
    x, f = w.stokes_uniform(500, seed=57)
    f = f[0] + np.array([0.5, 0.0, 0.0]) / 500  # a net force: allowed for the TP velocity, not for the pressure
    with pytest.raises(pk.PKIFMMError) as e:
        _plan_eval(pk.STOKES_PRESSURE, 7, x, f, 6)
    assert e.value.code == -3
