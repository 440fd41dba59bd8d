"""Many independent problems in one evaluation (one forest, one root per
problem): every problem's result equals its own evaluation and the oracle."""

import numpy as np
import pytest

import oracle
from gpu_util import rel_l2, run
from paper_1705_02043_gb300 import workloads as w
import paper_1705_02043_gb300 as pk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cache(tmp_path_factory):
    return str(tmp_path_factory.mktemp("opcache_batched"))


def _batched(kernel, periodic, x, d, off, p, leaf, precision=0, depth=10, nrhs=1, cache_dir=None):
    import torch
    k = 1 if kernel == 0 else 3
    dev = torch.device("cuda:0")
    plan = pk.PeriodicKIFMM(kernel, periodic, (0.0, 0.0, 0.0), 1.0, p, 2, leaf, depth, precision, nrhs, cache_dir)
    ts = torch.tensor(x, device=dev).contiguous()
    td = torch.tensor(np.asarray(d, np.float64).reshape(nrhs, len(x), k), device=dev).contiguous()
    out = plan.evaluate_batched(off, off, ts, td, ts)
    torch.cuda.synchronize()
    st = plan.tree_stats()
    plan.close()
    return out.cpu().numpy(), st


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_laplace_tp_matches_single_and_oracle(precision, cache):
    sizes = [700, 40, 2500, 1, 1300, 0, 900]
    x, q, off = w.multi_laplace_tp(len(sizes), seed=40, sizes=sizes)
    q[off[3]] = 0.0  # a one-point problem is neutral only with zero charge
    u, st = _batched(0, 7, x, q, off, p=8, leaf=32, precision=precision, cache_dir=cache)
    nbox = 0
    for j in range(len(sizes)):
        a, b = off[j], off[j + 1]
        if b == a:
            continue
        if b - a == 1:
            assert abs(u[0, a, 0]) < 1e-14
            continue
        one, plan = run(0, 7, x[a:b], q[a:b], x[a:b], p=8, leaf=32, precision=precision, cache_dir=cache,
                        return_plan=True)
        nbox += plan.tree_stats()[0]
        plan.close()
        ref = oracle.laplace_tp(x[a:b], q[a:b], x[a:b])
        if precision == 0:
            assert rel_l2(u[0, a:b, 0], one) < 1e-12
            assert rel_l2(u[0, a:b, 0], ref) < 1e-6
        else:
            assert rel_l2(u[0, a:b, 0], one) < 2e-5
            assert rel_l2(u[0, a:b, 0], ref) < 5e-5
    # the forest is the union of the problems' trees (empty problems keep a root)
    assert st[0] == nbox + sum(1 for j in range(len(sizes)) if off[j + 1] - off[j] <= 1)


def test_batched_stokes_dp_and_free(cache):
    for periodic in (3, 0):
        sizes = [800, 1500, 300]
        xs, fs = [], []
        for i, m in enumerate(sizes):
            xi, fi = w.stokes_uniform(m, seed=50 + i)
            xs.append(xi)
            fs.append(fi[0])
        x, f = np.concatenate(xs), np.concatenate(fs)
        off = np.concatenate([[0], np.cumsum(sizes)])
        u, _ = _batched(1, periodic, x, f, off, p=8, leaf=30, cache_dir=cache)
        for j in range(len(sizes)):
            a, b = off[j], off[j + 1]
            one = run(1, periodic, x[a:b], f[a:b], x[a:b], p=8, leaf=30, cache_dir=cache)
            assert rel_l2(u[0, a:b], one) < 1e-12


def test_batched_neutrality_is_per_problem(cache):
    x, q, off = w.multi_laplace_tp(3, seed=60, sizes=[200, 300, 250])
    q[off[1]] += 0.25  # problem 1 carries +0.25 ...
    q[off[2]] -= 0.25  # ... problem 2 -0.25: the total is still neutral
    with pytest.raises(pk.PKIFMMError) as e:
        _batched(0, 7, x, q, off, p=4, leaf=32, cache_dir=cache)
    assert e.value.name == "NOT_NEUTRAL"


def test_batched_bad_offsets(cache):
    x, q, off = w.multi_laplace_tp(2, seed=61, sizes=[100, 100])
    bad = off.copy()
    bad[1] = 150
    bad[2] = 120  # decreasing
    with pytest.raises(pk.PKIFMMError) as e:
        _batched(0, 7, x, q, bad, p=4, leaf=32, cache_dir=cache)
    assert e.value.name == "INVALID_ARG"


def test_autotune_leaf_picks_a_candidate(cache):
    import torch
    x, q, off = w.multi_laplace_tp(6, seed=62, lo=500, hi=4000)
    dev = torch.device("cuda:0")
    plan = pk.PeriodicKIFMM(0, 7, (0.0, 0.0, 0.0), 1.0, 6, 2, 32, 10, 0, 1, cache)
    ts = torch.tensor(x, device=dev).contiguous()
    td = torch.tensor(q[None, :, None], device=dev).contiguous()
    best, ms = plan.autotune_leaf(off, off, ts, td, ts, candidates=(16, 40, 96), reps=1)
    assert best in (16, 40, 96) and np.all(ms > 0) and ms[[16, 40, 96].index(best)] == ms.min()
    u = plan.evaluate_batched(off, off, ts, td, ts).cpu().numpy()
    plan.close()
    v, _ = _batched(0, 7, x, q, off, p=6, leaf=best, cache_dir=cache)
    # the tuned plan is the plan with that leaf size (up to the order of atomic sums)
    assert np.max(np.abs(u - v)) < 1e-12 * np.max(np.abs(v))
