"""Small named graphs with known triangle counts (edge lists, int32).

Every function returns ``(src, dst, n)``: numpy int32 arrays listing each
undirected edge once, plus the vertex count.  The triangle counts these
graphs are known to have are stated in the tests, not here: this module only
builds inputs.
"""
from __future__ import annotations

import itertools

import numpy as np


def _out(pairs, n):
    if len(pairs) == 0:
        z = np.zeros(0, np.int32)
        return z, z.copy(), n
    a = np.asarray(pairs, dtype=np.int64)
    return a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), n


def complete(n: int):
    """K_n."""
    iu = np.triu_indices(n, 1)
    return iu[0].astype(np.int32), iu[1].astype(np.int32), n


def complete_bipartite(a: int, b: int):
    """K_{a,b}: parts {0..a-1} and {a..a+b-1}."""
    return _out([(i, a + j) for i in range(a) for j in range(b)], a + b)


def star(k: int):
    """Hub 0 joined to k leaves."""
    return _out([(0, i) for i in range(1, k + 1)], k + 1)


def path(n: int):
    return _out([(i, i + 1) for i in range(n - 1)], n)


def cycle(n: int):
    """C_n for n >= 3."""
    return _out([(i, (i + 1) % n) for i in range(n)], n)


def wheel(k: int):
    """Hub 0 joined to every vertex of a rim cycle 1..k (k >= 3)."""
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
    spokes = [(0, 1 + i) for i in range(k)]
    return _out(rim + spokes, k + 1)


def friendship(k: int):
    """F_k: k triangles sharing the single vertex 0."""
    pairs = []
    for i in range(k):
        a, b = 1 + 2 * i, 2 + 2 * i
        pairs += [(0, a), (0, b), (a, b)]
    return _out(pairs, 2 * k + 1)


def hypercube(d: int):
    """Q_d on 2**d vertices; bipartite."""
    n = 1 << d
    return _out([(v, v ^ (1 << j)) for v in range(n) for j in range(d) if v < v ^ (1 << j)], n)


def random_tree(n: int, seed: int):
    """Uniform random recursive tree: vertex i>0 attaches to one of 0..i-1."""
    rng = np.random.default_rng(seed)
    return _out([(i, int(rng.integers(0, i))) for i in range(1, n)], n)


def grid(rows: int, cols: int):
    """rows x cols grid graph; bipartite."""
    idx = lambda r, c: r * cols + c
    pairs = []
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols:
                pairs.append((idx(r, c), idx(r, c + 1)))
            if r + 1 < rows:
                pairs.append((idx(r, c), idx(r + 1, c)))
    return _out(pairs, rows * cols)


def disjoint_union(*graphs):
    """Vertex-disjoint union; ids of each part are shifted past the previous ones."""
    srcs, dsts, off = [], [], 0
    for s, d, n in graphs:
        srcs.append(s.astype(np.int64) + off)
        dsts.append(d.astype(np.int64) + off)
        off += n
    return (np.concatenate(srcs).astype(np.int32), np.concatenate(dsts).astype(np.int32), off)


def complete_with_tree(n: int, tail: int, seed: int):
    """K_n with a random tree of `tail` extra vertices hanging off it."""
    rng = np.random.default_rng(seed)
    pairs = list(itertools.combinations(range(n), 2))
    for i in range(n, n + tail):
        pairs.append((i, int(rng.integers(0, i))))
    return _out(pairs, n + tail)


def random_multigraph(n: int, m: int, seed: int, loops: bool = True):
    """m uniform pairs with repeats, both directions and (optionally) loops."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, max(n, 1), m, dtype=np.int64)
    d = rng.integers(0, max(n, 1), m, dtype=np.int64)
    if not loops:
        keep = s != d
        s, d = s[keep], d[keep]
    return s.astype(np.int32), d.astype(np.int32), n


def gnp(n: int, p: float, seed: int):
    """G(n, p) with each edge listed once."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return iu[0][keep].astype(np.int32), iu[1][keep].astype(np.int32), n
