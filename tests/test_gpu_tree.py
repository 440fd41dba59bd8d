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
