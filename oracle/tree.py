"""Oracle (test infrastructure only): definitional adaptive octree and the
U/V/W/X interaction lists of kernel-independent FMM on a periodic box.

Sec. 2.2 builds an adaptive octree of B0 with at most s points per leaf and
copies it into the adjacent periodic images; the near field N^{B0} of B0
holds the images within one layer.  The paper defers the list definitions to
the original KIFMM; this module states them from their definitions and
evaluates them by brute force over all pairs of boxes (O(B^2), small trees
only).  Shifts p in {-1,0,1}^3 (zero on free axes) name the periodic image
of a source box: the pair (A, p) means the region A + p.

Readings taken (the paper is silent on them):
* points are normalised x' = (x - lo)/L; periodic coordinates are wrapped
  with x' - floor(x') (a result of exactly 1.0 becomes 0.0);
* the cell of a point at depth D is floor(x' * 2^D) per axis;
* a box splits while it holds more than s sources or more than s targets
  and its level is below depth_max; empty children are not created;
* U(B), B a leaf:  leaves A with A+p adjacent to B, plus B itself;
* V(B):  same-level boxes A+p, children of a colleague (adjacent or equal
  same-level box) of parent(B), not adjacent to B;
* W(B), B a leaf:  boxes A+p finer than B, not adjacent to B, whose parent
  (+p) is adjacent to B;
* X(B):  leaves A+p coarser than B, adjacent to parent(B), not adjacent to B
  (so that B is in W(A) with the opposite shift).
"Adjacent" means the closed boxes touch but their interiors are disjoint.
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


def normalise(x, lo, L, periodic_axes):
    """Map points to the unit box; wrap periodic axes.  Returns (x', ok)."""
    xp = (np.asarray(x, dtype=np.float64) - np.asarray(lo, dtype=np.float64)) / L
    ok = True
    for a in range(3):
        if periodic_axes >> a & 1:
            c = xp[:, a] - np.floor(xp[:, a])
            xp[:, a] = np.where(c >= 1.0, 0.0, c)
        elif len(xp) and ((xp[:, a] < 0.0).any() or (xp[:, a] >= 1.0).any()):
            ok = False
    return xp, ok


def cells(xp, depth):
    return np.minimum(np.floor(xp * float(2 ** depth)).astype(np.int64), 2 ** depth - 1)


@dataclass
class Box:
    level: int
    pos: tuple
    src: list = field(default_factory=list)
    trg: list = field(default_factory=list)
    children: list = field(default_factory=list)
    parent: "int | None" = None

    @property
    def is_leaf(self):
        return not self.children


def build(src_xp, trg_xp, leaf_max, depth_max):
    """Adaptive octree by recursive splitting; boxes listed level by level in
    Morton order of their children (octant index c = cx + 2 cy + 4 cz).  A
    child takes the parent's points whose cell at the child's level is the
    child's position (index lists kept in input order)."""
    cs, ct = cells(src_xp, depth_max), cells(trg_xp, depth_max)
    boxes = [Box(0, (0, 0, 0), list(range(len(cs))), list(range(len(ct))))]
    level = [0]
    while level:
        nxt = []
        for bi in level:
            b = boxes[bi]
            if b.level >= depth_max or (len(b.src) <= leaf_max and len(b.trg) <= leaf_max):
                continue
            sh = depth_max - b.level - 1
            bs, bt = np.asarray(b.src, dtype=np.int64), np.asarray(b.trg, dtype=np.int64)
            cells_s = cs[bs] >> sh if len(bs) else np.zeros((0, 3), np.int64)
            cells_t = ct[bt] >> sh if len(bt) else np.zeros((0, 3), np.int64)
            for c in range(8):
                off = (c & 1, c >> 1 & 1, c >> 2 & 1)
                pos = tuple(2 * b.pos[a] + off[a] for a in range(3))
                s = bs[(cells_s == np.array(pos)).all(axis=1)].tolist()
                t = bt[(cells_t == np.array(pos)).all(axis=1)].tolist()
                if not s and not t:
                    continue
                boxes.append(Box(b.level + 1, pos, s, t, [], bi))
                b.children.append(len(boxes) - 1)
                nxt.append(len(boxes) - 1)
        level = nxt
    return boxes


def shifts(periodic_axes):
    rng = [(-1, 0, 1) if periodic_axes >> a & 1 else (0,) for a in range(3)]
    return list(itertools.product(*rng))


def _span(box, p, lm):
    """Integer interval [lo, hi] per axis of box + p at level lm >= box.level."""
    f = 1 << (lm - box.level)
    lo = [(box.pos[a] + p[a] * (1 << box.level)) * f for a in range(3)]
    return lo, [v + f for v in lo]


def touch(A, p, B):
    lm = max(A.level, B.level)
    alo, ahi = _span(A, p, lm)
    blo, bhi = _span(B, (0, 0, 0), lm)
    t = all(alo[a] <= bhi[a] and blo[a] <= ahi[a] for a in range(3))
    inner = all(alo[a] < bhi[a] and blo[a] < ahi[a] for a in range(3))
    return t, inner


def adjacent(A, p, B):
    t, inner = touch(A, p, B)
    return t and not inner


def lists(boxes, periodic_axes):
    """Brute-force U, V, W, X lists: dict name -> {target box: set((src, p))}."""
    P = shifts(periodic_axes)
    nb = len(boxes)
    U = {i: set() for i in range(nb)}
    V = {i: set() for i in range(nb)}
    W = {i: set() for i in range(nb)}
    X = {i: set() for i in range(nb)}
    for bi, B in enumerate(boxes):
        for ai, A in enumerate(boxes):
            for p in P:
                adj = adjacent(A, p, B)
                if B.is_leaf and A.is_leaf and (adj or (ai == bi and p == (0, 0, 0))):
                    U[bi].add((ai, p))
                if B.parent is not None and A.level == B.level and A.parent is not None:
                    pa, pb = boxes[A.parent], boxes[B.parent]
                    t, _ = touch(pa, p, pb)
                    if t and not adj and not (ai == bi and p == (0, 0, 0)):
                        V[bi].add((ai, p))
                if B.is_leaf and A.level > B.level and not adj:
                    if adjacent(boxes[A.parent], p, B):
                        W[bi].add((ai, p))
                if B.parent is not None and A.is_leaf and A.level < B.level and not adj:
                    if adjacent(A, p, boxes[B.parent]):
                        X[bi].add((ai, p))
    return {"U": U, "V": V, "W": W, "X": X}


def _intersects(A, p, lo, hi, lev):
    """Does the closed region A + p meet the closed cube [lo, hi]^3 given in
    integer coordinates of level `lev` (lev >= A.level)?"""
    alo, ahi = _span(A, p, lev)
    return all(alo[a] <= hi[a] and lo[a] <= ahi[a] for a in range(3))


def lists_local(boxes, periodic_axes, targets=None):
    """The same U, V, W, X lists as ``lists`` (same predicates, term by term),
    with the source candidates of a target box B limited to the boxes A + p
    that meet R(B): parent(B) grown by one parent width on every side (B
    grown by its own width for a root).  Every list pairs B with boxes that
    meet R(B): a U source touches B; a W source lies in a box no larger than
    B that touches B; a V source lies in a box that touches parent(B) and is
    no larger than it; an X source touches parent(B).  Candidates are
    found by descending from the roots into the children that still meet
    R(B) (a box that misses R(B) has no child that meets it).  ``targets``
    restricts the target boxes (default: all)."""
    P = shifts(periodic_axes)
    nb = len(boxes)
    tg = range(nb) if targets is None else targets
    out = {n: {i: set() for i in tg} for n in "UVWX"}
    roots = [i for i, b in enumerate(boxes) if b.parent is None]
    lev = max(b.level for b in boxes) + 1          # fine enough for every box
    for bi in tg:
        B = boxes[bi]
        R = boxes[B.parent] if B.parent is not None else B
        f = 1 << (lev - R.level)
        lo = [R.pos[a] * f - f for a in range(3)]
        hi = [R.pos[a] * f + 2 * f for a in range(3)]
        for p in P:
            stack = [r for r in roots if _intersects(boxes[r], p, lo, hi, lev)]
            while stack:
                ai = stack.pop()
                A = boxes[ai]
                adj = adjacent(A, p, B)
                if B.is_leaf and A.is_leaf and (adj or (ai == bi and p == (0, 0, 0))):
                    out["U"][bi].add((ai, p))
                if B.parent is not None and A.level == B.level and A.parent is not None:
                    pa, pb = boxes[A.parent], boxes[B.parent]
                    t, _ = touch(pa, p, pb)
                    if t and not adj and not (ai == bi and p == (0, 0, 0)):
                        out["V"][bi].add((ai, p))
                if B.is_leaf and A.level > B.level and not adj:
                    if adjacent(boxes[A.parent], p, B):
                        out["W"][bi].add((ai, p))
                if B.parent is not None and A.is_leaf and A.level < B.level and not adj:
                    if adjacent(A, p, boxes[B.parent]):
                        out["X"][bi].add((ai, p))
                stack.extend(c for c in A.children if _intersects(boxes[c], p, lo, hi, lev))
    return out


def ancestors(boxes, i):
    out = [i]
    while boxes[out[-1]].parent is not None:
        out.append(boxes[out[-1]].parent)
    return out


def coverage_counts(boxes, L, periodic_axes):
    """For every (target leaf B, source leaf A, shift p) count the list routes
    that carry A+p's sources to B's targets: U(B); V(B') with A' (B', A'
    ancestors-or-self); W(B) with A' ancestor-or-self of A; X(B') with B'
    ancestor-or-self of B.  KIFMM is exact in its bookkeeping only if every
    count is 1 (the root periodic operator takes the images beyond one layer).
    """
    P = shifts(periodic_axes)
    leaves = [i for i, b in enumerate(boxes) if b.is_leaf]
    counts = {}
    for b in leaves:
        anc_b = ancestors(boxes, b)
        for a in leaves:
            anc_a = ancestors(boxes, a)
            for p in P:
                n = int((a, p) in L["U"][b])
                n += sum((a2, p) in L["V"][b2] for b2 in anc_b for a2 in anc_a)
                n += sum((a2, p) in L["W"][b] for a2 in anc_a)
                n += sum((a, p) in L["X"][b2] for b2 in anc_b)
                counts[(b, a, p)] = n
    return counts
