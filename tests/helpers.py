"""Independent reference computations used to pin the oracle.

None of these share code with the oracle or with the GPU library: they are
the textbook definitions (all triples; traces of adjacency-matrix powers)
written directly in numpy.
"""
from __future__ import annotations

import itertools

import numpy as np


def simple_adjacency(src, dst, n: int) -> np.ndarray:
    """0/1 int64 adjacency matrix of the simple undirected graph the pairs
    describe (self-loops dropped, repeats and directions collapsed)."""
    a = np.zeros((n, n), np.int64)
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    a[s[keep], d[keep]] = 1
    a[d[keep], s[keep]] = 1
    return a


def brute_force(src, dst, n: int):
    """Triangles by checking every vertex triple (n small)."""
    a = simple_adjacency(src, dst, n)
    T = 0
    t = np.zeros(n, np.int64)
    for i, j, k in itertools.combinations(range(n), 3):
        if a[i, j] and a[j, k] and a[i, k]:
            T += 1
            t[i] += 1
            t[j] += 1
            t[k] += 1
    return T, t


def trace_cubed(src, dst, n: int):
    """T = trace(A^3) / 6 and t(v) = (A^3)_vv / 2 in exact int64."""
    a = simple_adjacency(src, dst, n)
    a3 = a @ a @ a
    return int(np.trace(a3)) // 6, np.diag(a3) // 2


def sparse_counts(src, dst, n: int):
    """T and t(v) from (A @ A) * A with scipy sparse integer matrices."""
    import scipy.sparse as sp

    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    rows = np.concatenate([s[keep], d[keep]])
    cols = np.concatenate([d[keep], s[keep]])
    a = sp.coo_matrix((np.ones(len(rows), np.int64), (rows, cols)), shape=(n, n)).tocsr()
    a.data[:] = 1  # collapse repeats
    a.sum_duplicates()
    a.data[:] = 1
    paths = (a @ a).multiply(a)
    per_vertex = np.asarray(paths.sum(axis=1)).ravel() // 2
    return int(paths.sum()) // 6, per_vertex.astype(np.int64)


def simple_degrees(src, dst, n: int) -> np.ndarray:
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    a, b = np.minimum(s[keep], d[keep]), np.maximum(s[keep], d[keep])
    key = np.unique(a * max(n, 1) + b)
    deg = np.zeros(n, np.int64)
    np.add.at(deg, key // max(n, 1), 1)
    np.add.at(deg, key % max(n, 1), 1)
    return deg
