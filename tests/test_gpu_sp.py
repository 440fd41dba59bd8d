"""Singly periodic Stokes CUDA path vs the oracle (image sum with a
closed-form Euler-Maclaurin tail); zero net force."""

import numpy as np
import pytest

import oracle
from gpu_util import rel_l2, run
from paper_1705_02043_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cache(tmp_path_factory):
    return str(tmp_path_factory.mktemp("opcache_sp"))


@pytest.mark.parametrize("axis,p,tol", [(0, 10, 2e-7), (2, 12, 1e-8)])
def test_stokes_sp_fp64(axis, p, tol, cache):
    x, f = w.stokes_uniform(2500, seed=70 + axis)
    u = run(1, 1 << axis, x, f[0], x, p=p, leaf=40, cache_dir=cache)
    ref = oracle.stokes_sp(x, f[0], x, axis=axis)
    e = rel_l2(u, ref)
    print(f"stokes SP axis {axis} p={p} rel_l2 {e:.3e}")
    assert e < tol


def test_stokes_sp_error_falls_with_p_and_mixed(cache):
    x, f = w.stokes_uniform(4000, seed=73)
    ref = oracle.stokes_sp(x, f[0], x, axis=1)
    errs = [rel_l2(run(1, 2, x, f[0], x, p=p, leaf=40, cache_dir=cache), ref) for p in (4, 6, 8)]
    print("stokes SP errors p=4,6,8", errs)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-5
    em = rel_l2(run(1, 2, x, f[0], x, p=8, leaf=40, precision=1, cache_dir=cache), ref)
    print("stokes SP mixed p=8", em)
    assert em < 2e-5
