"""GPU octree and interaction lists vs the definitional oracle: bit-exact.

The box set (level, position), each box's source and target index sets, and
every list as a set of (target box, source box, periodic shift) must equal
the oracle's brute-force construction."""

import numpy as np
import pytest

from gpu_util import run
from oracle import tree
from paper_1705_02043_gb300 import workloads as w
import paper_1705_02043_gb300 as pk

pytestmark = pytest.mark.gpu


def _gpu_tree(plan, S, T):
    t = pk.pkifmm_tree_export(plan.handle, S, T)
    keys = [(int(l), tuple(int(v) for v in p)) for l, p in zip(t["level"], t["pos"])]
    lists = {}
    for name in "UVWX":
        ptr, box, sh = pk.pkifmm_list_export(plan.handle, name)
        s = set()
        for b in range(len(keys)):
            for e in range(ptr[b], ptr[b + 1]):
                s.add((keys[b], keys[box[e]], tuple(int(v) for v in sh[e])))
        lists[name] = s
    return t, keys, lists


def _oracle_tree(src, trg, periodic, leaf, depth):
    sp, _ = tree.normalise(src, [0, 0, 0], 1.0, periodic)
    tp, _ = tree.normalise(trg, [0, 0, 0], 1.0, periodic)
    boxes = tree.build(sp, tp, leaf, depth)
    L = tree.lists(boxes, periodic)
    keys = [(b.level, b.pos) for b in boxes]
    lists = {n: {(keys[t], keys[a], p) for t, v in L[n].items() for a, p in v} for n in "UVWX"}
    return boxes, keys, lists


@pytest.mark.parametrize("periodic", [7, 3, 1, 4, 0])
def test_tree_and_lists_bit_exact(periodic):
    trg, _ = w.clustered_slab(400, seed=21, nclusters=4, sigma=0.05, zlo=0.0, zhi=1.0, kdim=1)
    src = w.uniform_points(150, seed=22)
    q = np.ones(len(src)) * np.where(np.arange(len(src)) % 2 == 0, 1.0, -1.0)
    leaf, depth = 6, 6
    _, plan = run(0, periodic, src, q, trg, p=4, leaf=leaf, depth=depth, return_plan=True)
    t, gk, gl = _gpu_tree(plan, len(src), len(trg))
    plan.close()
    boxes, ok, ol = _oracle_tree(src, trg, periodic, leaf, depth)
    assert sorted(gk) == sorted(ok)
    idx = {k: i for i, k in enumerate(ok)}
    for b, k in enumerate(gk):
        ob = boxes[idx[k]]
        s0, s1 = t["src_range"][b]
        t0, t1 = t["trg_range"][b]
        assert set(t["src_perm"][s0:s1].tolist()) == set(ob.src)
        assert set(t["trg_perm"][t0:t1].tolist()) == set(ob.trg)
    # the permutation is a stable sort by Morton key at depth D
    for x, perm in ((src, t["src_perm"]), (trg, t["trg_perm"])):
        xp, _ = tree.normalise(x, [0, 0, 0], 1.0, periodic)
        c = tree.cells(xp, depth)
        key = np.zeros(len(c), np.int64)
        for bit in range(depth):
            for a in range(3):
                key |= ((c[:, a] >> bit) & 1) << (3 * bit + a)
        assert np.array_equal(perm, np.argsort(key, kind="stable"))
    for name in "UVWX":
        assert gl[name] == ol[name], name
    assert len(gl["W"]) > 0 and len(gl["X"]) > 0


def test_uniform_tree_v_counts():
    g = (np.arange(8) + 0.5) / 8
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    q = np.where(np.arange(len(pts)) % 2 == 0, 1.0, -1.0)
    _, plan = run(0, 7, pts, q, pts, p=4, leaf=1, depth=3, return_plan=True)
    st = plan.tree_stats()
    plan.close()
    nbox, nleaf, depth = st[0], st[1], st[2]
    assert (nbox, nleaf, depth) == (1 + 8 + 64 + 512, 512, 3)
    assert st[4] == 189 * (8 + 64 + 512)     # V entries
    assert st[3] == 27 * 512                  # U entries
    assert st[5] == 0 and st[6] == 0          # no W / X on a uniform tree


def _morton_perm(x, periodic, depth):
    """Stable argsort of the oracle's Morton keys at `depth` (octant bits x = 1, y = 2, z = 4)."""
    xp, _ = tree.normalise(x, [0, 0, 0], 1.0, periodic)
    c = tree.cells(xp, depth)
    key = np.zeros(len(c), np.int64)
    for bit in range(depth):
        for a in range(3):
            key |= ((c[:, a] >> bit) & 1) << (3 * bit + a)
    return np.argsort(key, kind="stable")


def _evaluate_for_tree(src, trg, periodic, leaf, depth):
    """One FP64 Laplace evaluation (p = 4) whose plan keeps its tree; trg None:
    the targets are the sources (one tensor, sorted once)."""
    import torch
    dev = torch.device("cuda:0")
    q = w.make_neutral(np.where(np.arange(len(src)) % 2 == 0, 1.0, -1.0))
    plan = pk.PeriodicKIFMM(pk.LAPLACE, periodic, (0.0, 0.0, 0.0), 1.0, 4, 2, leaf, depth, pk.FP64, 1)
    ts = torch.tensor(src, device=dev)
    tt = ts if trg is None else torch.tensor(trg, device=dev)
    plan.evaluate(ts, torch.tensor(q[None, :, None], device=dev), tt)
    torch.cuda.synchronize()
    return plan


def _check_boxes(t, gk, boxes, ok):
    assert sorted(gk) == sorted(ok)
    idx = {k: i for i, k in enumerate(ok)}
    for b, k in enumerate(gk):
        ob = boxes[idx[k]]
        s0, s1 = t["src_range"][b]
        t0, t1 = t["trg_range"][b]
        assert np.array_equal(np.sort(t["src_perm"][s0:s1]), np.asarray(ob.src, dtype=np.int64))
        assert np.array_equal(np.sort(t["trg_perm"][t0:t1]), np.asarray(ob.trg, dtype=np.int64))


@pytest.mark.parametrize("periodic,same", [(7, True), (3, False)])
def test_deep_clustered_tree_and_lists_bit_exact(periodic, same):
    """24,000 points in 16 tight clusters, leaf 16, depth_max 12 (the tree
    reaches level 10): several radix tiles of 4,096 keys, W and X lists;
    every box, point set, list entry and both permutations equal the
    oracle's."""
    src, _ = w.clustered_slab(24000, seed=41, nclusters=16, sigma=0.004, zlo=0.0, zhi=1.0, kdim=1)
    trg = None if same else w.clustered_slab(20000, seed=42, nclusters=12, sigma=0.004, zlo=0.0, zhi=1.0,
                                             kdim=1)[0]
    leaf, depth = 16, 12
    plan = _evaluate_for_tree(src, trg, periodic, leaf, depth)
    t, gk, gl = _gpu_tree(plan, len(src), len(src) if same else len(trg))
    plan.close()
    trg_pts = src if same else trg
    sp, _ = tree.normalise(src, [0, 0, 0], 1.0, periodic)
    tp, _ = tree.normalise(trg_pts, [0, 0, 0], 1.0, periodic)
    boxes = tree.build(sp, tp, leaf, depth)
    assert max(b.level for b in boxes) >= 9
    ok = [(b.level, b.pos) for b in boxes]
    _check_boxes(t, gk, boxes, ok)
    assert np.array_equal(t["src_perm"], _morton_perm(src, periodic, depth))
    assert np.array_equal(t["trg_perm"], _morton_perm(trg_pts, periodic, depth))
    L = tree.lists_local(boxes, periodic)
    for name in "UVWX":
        want = {(ok[b], ok[a], p) for b, v in L[name].items() for a, p in v}
        assert gl[name] == want, name
    assert len(gl["W"]) > 0 and len(gl["X"]) > 0


def test_large_tree_with_wrapped_images():
    """2^17 clustered points, a seventh of them moved by whole periods (the
    library wraps them), depth 12: the permutation equals the stable argsort
    of the oracle's keys, the box set and point sets equal the oracle's, and
    the lists of 300 seeded target boxes equal the oracle's."""
    n, leaf, depth, periodic = 1 << 17, 32, 12, 7
    x, _ = w.clustered_slab(n, seed=43, nclusters=32, sigma=0.004, zlo=0.0, zhi=1.0, kdim=1)
    x[::7] += np.array([1.0, -2.0, 1.0])
    plan = _evaluate_for_tree(x, None, periodic, leaf, depth)
    t = pk.pkifmm_tree_export(plan.handle, n, n)
    gk = [(int(l), tuple(int(v) for v in p)) for l, p in zip(t["level"], t["pos"])]
    glist = {name: pk.pkifmm_list_export(plan.handle, name) for name in "UVWX"}
    plan.close()
    perm = _morton_perm(x, periodic, depth)
    assert np.array_equal(t["src_perm"], perm) and np.array_equal(t["trg_perm"], perm)
    xp, _ = tree.normalise(x, [0, 0, 0], 1.0, periodic)
    boxes = tree.build(xp, xp, leaf, depth)
    assert max(b.level for b in boxes) >= 10
    ok = [(b.level, b.pos) for b in boxes]
    _check_boxes(t, gk, boxes, ok)
    sub = sorted(np.random.default_rng(0).choice(len(boxes), 300, replace=False).tolist())
    L = tree.lists_local(boxes, periodic, targets=sub)
    gidx = {k: i for i, k in enumerate(gk)}
    for name in "UVWX":
        ptr, box, sh = glist[name]
        for b in sub:
            g = gidx[ok[b]]
            got = {(gk[box[e]], tuple(int(v) for v in sh[e])) for e in range(ptr[g], ptr[g + 1])}
            assert got == {(ok[a], p) for a, p in L[name][b]}, (name, ok[b])
