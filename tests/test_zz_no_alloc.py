"""The allocation-free Morton ordering entry point (for callers that cannot
call cudaMalloc: a device whose memory another framework's pool owns, a
real-time loop that forbids allocation after start-up, code where CUDA
allocation calls are not permitted) must give the same permutation as the
ordering the full evaluation computes for its sources, on consecutive calls
that reuse its fixed scratch.  Collected last so a failure here comes after
every other test has run."""

import ctypes

import numpy as np
import pytest

import paper_1705_02043_gb300 as pk
from paper_1705_02043_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def _reference_perm(x, lo, L, periodic, depth):
    """Sources' sorted order from the existing entry points (evaluate + export)."""
    import torch
    plan = pk.PeriodicKIFMM(pk.LAPLACE, periodic, lo, L, p=4, leaf_max=1 << 20, depth_max=depth)
    dev = torch.device("cuda:0")
    tx = torch.tensor(x, device=dev)
    q = torch.zeros((1, len(x), 1), dtype=torch.float64, device=dev)
    plan.evaluate(tx, q, tx[:1].contiguous())
    torch.cuda.synchronize()
    perm = pk.pkifmm_tree_export(plan.handle, len(x), 1)["src_perm"]
    plan.close()
    return perm


def test_morton_order_noalloc_matches_evaluation_order():
    import torch
    dev = torch.device("cuda:0")
    lo, L = np.array([-1.0, 0.5, 2.0]), 3.0
    cases = [(100000, 7, 10, 1), (131072, 0, 12, 2)]  # two calls in a row, different inputs
    for n, periodic, depth, seed in cases:
        x = lo + L * w.uniform_points(n, seed=seed)
        if periodic:
            x[::7] += L * np.array([1.0, -2.0, 1.0])  # images along periodic axes are wrapped
        ref = _reference_perm(x, lo, L, periodic, depth)
        tx = torch.tensor(x, device=dev)
        perm = torch.full((n,), -1, dtype=torch.int32, device=dev)
        pk.pkifmm_morton_order_noalloc(n, tx, lo, L, periodic, depth, perm,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        got = perm.cpu().numpy().astype(np.int64)
        assert np.array_equal(got, ref)


def test_morton_order_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = 131073
    tx = torch.zeros((n, 3), dtype=torch.float64, device="cuda:0")
    perm = torch.zeros((n,), dtype=torch.int32, device="cuda:0")
    with pytest.raises(pk.PKIFMMError) as e:
        pk.pkifmm_morton_order_noalloc(n, tx, (0.0, 0.0, 0.0), 1.0, 7, 10, perm)
    assert e.value.name == "INVALID_ARG"
