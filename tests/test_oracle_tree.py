"""Pins for the definitional octree / interaction-list oracle.

The lists are checked against what the method needs of them: every
(target leaf, source leaf, periodic image within one layer) interaction is
carried by exactly one route (U, V, W or X, through ancestors), and on a
uniform full tree each box sees the textbook counts (27 adjacent boxes and
189 well-separated children of its parent's colleagues).
"""

import numpy as np
import pytest

from oracle import tree
from paper_1705_02043_gb300 import workloads as w


@pytest.mark.parametrize("periodic", [7, 3, 4, 0])
def test_every_interaction_covered_exactly_once(periodic):
    x, _ = w.clustered_slab(240, seed=11, nclusters=3, sigma=0.06, zlo=0.0, zhi=1.0, kdim=1)
    y = w.uniform_points(60, seed=12)
    xp, ok = tree.normalise(x, [0, 0, 0], 1.0, periodic)
    yp, _ = tree.normalise(y, [0, 0, 0], 1.0, periodic)
    assert ok
    boxes = tree.build(yp, xp, 7, 6)  # sources: uniform, targets: clustered
    L = tree.lists(boxes, periodic)
    counts = tree.coverage_counts(boxes, L, periodic)
    assert counts and set(counts.values()) == {1}
    # adaptive: the tree must have W/X work to be a meaningful check
    assert sum(len(v) for v in L["W"].values()) > 0
    assert sum(len(v) for v in L["X"].values()) > 0


def test_uniform_full_tree_counts_tp():
    # 8 points per level-2 cell, leaf cap 8 -> full uniform tree of depth 2
    g = (np.arange(4) + 0.5) / 4
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pts = np.concatenate([c + d for d in np.linspace(-0.1, 0.1, 8)[:, None] * np.array([[1, 0.3, 0.7]])])
    xp, _ = tree.normalise(pts, [0, 0, 0], 1.0, 7)
    boxes = tree.build(xp, xp, 8, 5)
    L = tree.lists(boxes, 7)
    leaves = [i for i, b in enumerate(boxes) if b.is_leaf]
    assert len(leaves) == 64 and all(boxes[i].level == 2 for i in leaves)
    assert all(len(L["U"][i]) == 27 for i in leaves)
    assert all(len(L["V"][i]) == 189 for i, b in enumerate(boxes) if b.level >= 1)
    assert all(len(L["W"][i]) == 0 and len(L["X"][i]) == 0 for i in range(len(boxes)))


def test_root_leaf_sees_its_images():
    xp = w.uniform_points(5, seed=1)
    boxes = tree.build(xp, xp, 10, 4)
    assert len(boxes) == 1
    for periodic, n in ((7, 27), (3, 9), (1, 3), (0, 1)):
        L = tree.lists(boxes, periodic)
        assert len(L["U"][0]) == n


def test_normalise_wraps_and_flags():
    x = np.array([[-0.25, 1.5, 0.5], [1.0, 0.0, 0.999]])
    xp, ok = tree.normalise(x, [0, 0, 0], 1.0, 3)
    assert ok and np.allclose(xp[:, :2], [[0.75, 0.5], [0.0, 0.0]])
    _, ok = tree.normalise(x, [0, 0, 0], 1.0, 1)
    assert not ok


@pytest.mark.parametrize("periodic", [7, 3, 1, 4, 0])
def test_local_search_equals_brute_force(periodic):
    """The candidate-pruned list builder returns exactly the brute-force lists
    (adaptive trees with W and X entries, sources and targets differing)."""
    x, _ = w.clustered_slab(300, seed=31, nclusters=3, sigma=0.05, zlo=0.0, zhi=1.0, kdim=1)
    y = w.uniform_points(120, seed=32)
    xp, _ = tree.normalise(x, [0, 0, 0], 1.0, periodic)
    yp, _ = tree.normalise(y, [0, 0, 0], 1.0, periodic)
    for src, trg, leaf in ((yp, xp, 6), (xp, xp, 4)):
        boxes = tree.build(src, trg, leaf, 6)
        full = tree.lists(boxes, periodic)
        local = tree.lists_local(boxes, periodic)
        for name in "UVWX":
            assert local[name] == full[name], name
        assert sum(len(v) for v in full["W"].values()) > 0 and sum(len(v) for v in full["X"].values()) > 0
    # a subset of target boxes gives those boxes' lists
    sub = list(range(0, len(boxes), 5))
    part = tree.lists_local(boxes, periodic, targets=sub)
    for name in "UVWX":
        assert part[name] == {b: full[name][b] for b in sub}


def test_local_search_root_leaf_images():
    xp = w.uniform_points(5, seed=1)
    boxes = tree.build(xp, xp, 10, 4)
    for periodic, n in ((7, 27), (3, 9), (1, 3), (0, 1)):
        assert len(tree.lists_local(boxes, periodic)["U"][0]) == n
