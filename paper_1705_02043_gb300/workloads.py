"""Seeded synthetic inputs shaped like the paper's test problems.

This module only draws points and densities; it holds none of the method's
arithmetic, so the tests, the benchmark and the oracle checks can all use it.
Every generator uses numpy's PCG64 with an explicit seed.

Densities that must be neutral (zero net charge / zero net force, the
compatibility condition of Eq. (compatcondition), Sec. 2.2) are quantised to
multiples of 2**-40 so that the last entry can be chosen to make the sum
exactly zero in binary64.
"""

from __future__ import annotations

import math

import numpy as np

_Q = 2.0 ** 40  # quantum for exactly-neutral densities


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_neutral(values: np.ndarray) -> np.ndarray:
    """Shift a [N] or [N][k] density to zero sum per component, exactly.

    Values are rounded to multiples of 2**-40; the mean is removed and the
    last entry absorbs the residual, so math.fsum of each component is 0.
    """
    v = np.array(values, dtype=np.float64, copy=True)
    squeeze = v.ndim == 1
    if v.shape[0] == 0:
        return v
    if squeeze:
        v = v[:, None]
    v = np.round(v * _Q) / _Q
    v -= np.round(v.mean(axis=0) * _Q) / _Q
    for c in range(v.shape[1]):
        v[-1, c] = -math.fsum(v[:-1, c])
        assert math.fsum(v[:, c]) == 0.0
    return v[:, 0] if squeeze else v


def uniform_points(n: int, seed: int, box: float = 1.0) -> np.ndarray:
    return _rng(seed).random((n, 3)) * box


def laplace_sp_uniform(n: int = 2000, seed: int = 0):
    """Laplace, singly periodic: N uniform points, charges U[-1,1], neutral."""
    rng = _rng(seed)
    x = rng.random((n, 3))
    q = make_neutral(rng.uniform(-1.0, 1.0, size=n))
    return x, q


def stokes_uniform(n: int, seed: int = 0, nrhs: int = 1, neutral: bool = True):
    """Stokes: N uniform points, forces N(0,1) per component, net force removed.

    Returns points [N][3] and forces [nrhs][N][3].
    """
    rng = _rng(seed)
    x = rng.random((n, 3))
    f = np.empty((nrhs, n, 3))
    for r in range(nrhs):
        g = rng.standard_normal((n, 3))
        f[r] = make_neutral(g) if neutral else g
    return x, f


def laplace_uniform(n: int, seed: int = 0, nrhs: int = 1):
    """Laplace: N uniform points, neutral charges U[-1,1]; charges [nrhs][N]."""
    rng = _rng(seed)
    x = rng.random((n, 3))
    q = np.empty((nrhs, n))
    for r in range(nrhs):
        q[r] = make_neutral(rng.uniform(-1.0, 1.0, size=n))
    return x, q


def clustered_slab(n: int, seed: int = 0, nclusters: int = 64, sigma: float = 0.02,
                   zlo: float = 0.0, zhi: float = 0.2, kdim: int = 3):
    """Points in Gaussian clusters inside a slab z in [zlo, zhi], x,y wrapped.

    Cluster centres: x,y uniform in [0,1), z uniform in [zlo+0.2w, zlo+0.8w]
    (w = zhi - zlo).  Each point's z is redrawn until it lies in [zlo, zhi).
    Densities: N(0,1) per component, made neutral.
    """
    rng = _rng(seed)
    w = zhi - zlo
    centres = np.column_stack([rng.random(nclusters), rng.random(nclusters),
                               zlo + w * (0.2 + 0.6 * rng.random(nclusters))])
    per = np.full(nclusters, n // nclusters)
    per[: n - per.sum()] += 1
    pts = []
    for c in range(nclusters):
        m = per[c]
        p = centres[c] + sigma * rng.standard_normal((m, 3))
        bad = (p[:, 2] < zlo) | (p[:, 2] >= zhi)
        while bad.any():
            p[bad, 2] = centres[c, 2] + sigma * rng.standard_normal(bad.sum())
            bad = (p[:, 2] < zlo) | (p[:, 2] >= zhi)
        pts.append(p)
    x = np.concatenate(pts)
    x[:, :2] -= np.floor(x[:, :2])
    x[:, :2] = np.where(x[:, :2] >= 1.0, 0.0, x[:, :2])
    d = make_neutral(rng.standard_normal((n, kdim)))
    return x, (d[:, 0] if kdim == 1 else d)


def chebyshev_grid(m: int = 97) -> np.ndarray:
    """Clenshaw-Curtis points c_i = (1 - cos(pi i/(m-1)))/2 as an m^3 grid.

    Sec. 3.3: the target grid of the Stokes accuracy tests (97^3 points).
    Ordering: i (x) slowest, k (z) fastest.
    """
    c = 0.5 * (1.0 - np.cos(np.pi * np.arange(m) / (m - 1)))
    g = np.stack(np.meshgrid(c, c, c, indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def lognormal_points(n: int, seed: int = 0, mu: float = 0.2, s: float = 0.5) -> np.ndarray:
    """Sec. 3.4 non-uniform points: each coordinate lognormal(mu, s), wrapped mod 1."""
    x = _rng(seed).lognormal(mu, s, size=(n, 3))
    x -= np.floor(x)
    return np.where(x >= 1.0, 0.0, x)


def madelung_1d():
    """Sec. 3.2: four alternating unit charges on the z axis line x=y=0.5.

    Returns (sources, charges, targets); the exact potential at both targets
    (the positive charges) is -8 ln 2 for unit period along z.
    """
    src = np.array([[0.5, 0.5, 0.125], [0.5, 0.5, 0.375],
                    [0.5, 0.5, 0.625], [0.5, 0.5, 0.875]])
    q = np.array([1.0, -1.0, 1.0, -1.0])
    trg = src[[0, 2]].copy()
    return src, q, trg


def two_forces():
    """Sec. 3.3: f1 at (0.7,0.6,0.5) = (1,2,3)/sqrt(14), f2 = -f1 at (0.2,0.8,0.7)."""
    f1 = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
    src = np.array([[0.7, 0.6, 0.5], [0.2, 0.8, 0.7]])
    return src, np.stack([f1, -f1])


def single_force():
    """Sec. 3.4: one force (1,2,3)/sqrt(14) at (0.7,0.6,0.4) (net force allowed in TP)."""
    return np.array([[0.7, 0.6, 0.4]]), (np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0))[None, :]


def multi_problem_sizes(nprob: int = 256, seed: int = 0, lo: int = 1024, hi: int = 65536):
    """Problem sizes log-uniform in [lo, hi] (rounded), one per problem."""
    rng = _rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=nprob))).astype(np.int64)


def multi_laplace_tp(nprob: int = 256, seed: int = 0, lo: int = 1024, hi: int = 65536, sizes=None):
    """Independent Laplace problems, concatenated: sizes log-uniform in [lo, hi]
    (or given), problem i uniform in the unit cube with neutral charges U[-1,1]
    drawn with seed + i.  Returns points [S][3], charges [S], CSR offsets [nprob+1]."""
    n = multi_problem_sizes(nprob, seed, lo, hi) if sizes is None else np.asarray(sizes, dtype=np.int64)
    xs, qs = [], []
    for i, m in enumerate(n):
        x, q = laplace_uniform(int(m), seed=seed + i)
        xs.append(x)
        qs.append(q[0])
    off = np.zeros(len(n) + 1, dtype=np.int64)
    off[1:] = np.cumsum(n)
    return np.concatenate(xs) if xs else np.zeros((0, 3)), np.concatenate(qs) if qs else np.zeros(0), off
