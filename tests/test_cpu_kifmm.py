"""The plain CPU KIFMM baseline against the oracle (host only).

The baseline is not on the GPU library's path; these tests make sure the
number bench.py reports beside the GPU run comes from a correct program."""

import numpy as np
import pytest

import oracle
from baseline import cpu_kifmm
from paper_1705_02043_gb300 import workloads as w


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("periodic,tol", [(7, 5e-6), (0, 2e-6)])
def test_stokes_p8(periodic, tol):
    x, f = w.stokes_uniform(3000, seed=3, nrhs=1)
    u, t, depth = cpu_kifmm.evaluate(1, periodic, 8, 64, x, f[0])
    idx = np.arange(0, 3000, 25)
    e = _rel(u[idx], oracle.periodic_sum(1, periodic, x, f[0], x[idx]))
    print(f"cpu kifmm stokes periodic {periodic} p=8 depth {depth}: {e:.2e}")
    assert depth >= 2 and e < tol


def test_laplace_tp_p6_needs_the_second_moment_constant():
    x, q = w.laplace_uniform(3000, seed=4)
    u, _, _ = cpu_kifmm.evaluate(0, 7, 6, 64, x, q[0])
    idx = np.arange(0, 3000, 25)
    e = _rel(u[idx], oracle.periodic_sum(0, 7, x, q[0], x[idx]))
    assert e < 2e-5


def test_bad_arguments():
    x = np.array([[0.5, 0.5, 1.0]])
    with pytest.raises(ValueError):
        cpu_kifmm.evaluate(1, 7, 8, 64, x, np.zeros((1, 3)))
    with pytest.raises(ValueError):
        cpu_kifmm.evaluate(1, 3, 8, 64, np.full((1, 3), 0.5), np.zeros((1, 3)))
