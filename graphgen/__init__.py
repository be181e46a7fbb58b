"""Seeded synthetic graph inputs (edge lists of int32 vertex ids).

Only inputs live here: nothing in this package orders, orients, sorts or
intersects adjacency lists.  Both the GPU library and the CPU oracle consume
these edge lists; neither imports the other.

The heavy generators are C (``graphgen.c``, SplitMix64 counter-based
randomness, deterministic for any thread count and host); ``families.py``
holds the small closed-form graphs used by the oracle's pins.

Named workloads (the paper evaluates on SNAP/DIMACS graphs, R-MAT Kronecker
graphs, Barabasi-Albert and Watts-Strogatz networks, Table 1; those datasets
are not available, so seeded synthetic graphs of the same families stand in):

  er16k     Erdos-Renyi n=16384, m=131072 distinct edges
  rmat20    R-MAT scale 20, 16,777,216 raw draws (a,b,c,d)=(.57,.19,.19,.05),
            permuted ids, self-loops and duplicates kept in the input
  rgg4m     random geometric graph, n=4,194,304, r=sqrt(32/(pi n))
  rmat24    R-MAT scale 24, draws until 180,000,000 distinct edges
  rmat22    R-MAT scale 22, draws until 45,000,000 distinct edges (profiling)
  ba200k    Barabasi-Albert n=200,000, 50 edges per new vertex (9,998,725)
  ws1m      Watts-Strogatz n=1,000,000, 25 neighbours on either side,
            rewiring probability 0.1 (25,000,000 pairs)
  batch4096 4096 graphs, half Erdos-Renyi, half R-MAT (a,b,c = .57,.19,.19),
            n log-uniform in [2^8, 2^18], mean degree uniform in [4, 64]
            (graph_batch(4096, 1005))
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_build", "libgraphgen.so")
_lib = None
_lock = threading.Lock()

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc (host code only, portable flags)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
             "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
            lib.gg_er.restype = ctypes.c_int64
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, i32p, i32p]
            lib.gg_rmat.restype = ctypes.c_int
            lib.gg_rmat_distinct.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                             i32p, i32p]
            lib.gg_rmat_distinct.restype = ctypes.c_int64
            lib.gg_rgg.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, i32p, i32p,
                                   ctypes.c_int64]
            lib.gg_rgg.restype = ctypes.c_int64
            lib.gg_rmat_graph.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                          i32p, i32p]
            lib.gg_rmat_graph.restype = ctypes.c_int64
            f64p = ctypes.POINTER(ctypes.c_double)
            lib.gg_rgg_point_coords.argtypes = [ctypes.c_int32, ctypes.c_uint64, f64p, f64p]
            lib.gg_rgg_point_coords.restype = None
            lib.gg_rgg_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gg_rgg_permutation.restype = None
            lib.gg_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p, i32p]
            lib.gg_ba.restype = ctypes.c_int64
            lib.gg_ws.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_uint64, i32p, i32p]
            lib.gg_ws.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def er(n: int, m: int, seed: int):
    """G(n, m): m distinct non-loop undirected edges, each listed once."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gg_er(n, m, seed, _ptr(src), _ptr(dst))
    if rc < 0:
        raise ValueError("gg_er(n=%d, m=%d) failed: %d" % (n, m, rc))
    return src, dst


def rmat(scale: int, draws: int, seed: int, abc=RMAT_ABC, permute: bool = True):
    """Raw R-MAT draws over 2**scale vertices (loops/duplicates kept)."""
    src = np.empty(draws, np.int32)
    dst = np.empty(draws, np.int32)
    rc = _load().gg_rmat(scale, draws, abc[0], abc[1], abc[2], seed, int(permute),
                         _ptr(src), _ptr(dst))
    if rc < 0:
        raise ValueError("gg_rmat failed: %d" % rc)
    return src, dst


def rmat_distinct(scale: int, m: int, seed: int, abc=RMAT_ABC):
    """R-MAT draws until m distinct non-loop undirected edges; each once."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gg_rmat_distinct(scale, m, abc[0], abc[1], abc[2], seed, _ptr(src), _ptr(dst))
    if rc < 0:
        raise ValueError("gg_rmat_distinct failed: %d" % rc)
    return src, dst


def rmat_graph(n: int, m: int, seed: int, abc=RMAT_ABC):
    """One R-MAT graph on n vertices (any n >= 2) with m distinct edges."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gg_rmat_graph(n, m, abc[0], abc[1], abc[2], seed, _ptr(src), _ptr(dst))
    if rc < 0:
        raise ValueError("gg_rmat_graph(n=%d, m=%d) failed: %d" % (n, m, rc))
    return src, dst


class GraphBatch:
    """Many graphs stored back to back: graph g has pairs
    src[edge_offsets[g]:edge_offsets[g+1]] (ids local to the graph) and
    vertex_counts[g] vertices; kinds[g] is 'er' or 'rmat'."""

    def __init__(self, src, dst, edge_offsets, vertex_counts, kinds, seeds):
        self.src, self.dst = src, dst
        self.edge_offsets = np.asarray(edge_offsets, np.int64)
        self.vertex_counts = np.asarray(vertex_counts, np.int32)
        self.kinds, self.seeds = list(kinds), list(seeds)

    def __len__(self):
        return len(self.vertex_counts)

    def graph(self, g):
        a, b = self.edge_offsets[g], self.edge_offsets[g + 1]
        return self.src[a:b], self.dst[a:b], int(self.vertex_counts[g])


def batch_params(count: int, seed: int, log2_n=(8, 18), degree=(4.0, 64.0)):
    """Seeded sizes of a batch: n log-uniform in [2^lo, 2^hi], mean degree
    uniform, m = floor(n d / 2) distinct edges; even g Erdos-Renyi, odd
    R-MAT."""
    rng = np.random.default_rng(seed)
    lo, hi = log2_n
    n = np.floor(np.exp2(lo + (hi - lo) * rng.random(count))).astype(np.int64)
    d = degree[0] + (degree[1] - degree[0]) * rng.random(count)
    m = np.floor(n * d / 2).astype(np.int64)
    m = np.minimum(m, n * (n - 1) // 4)  # keep well inside the simple-graph limit
    kinds = ["er" if g % 2 == 0 else "rmat" for g in range(count)]
    seeds = [int(seed) * 1_000_003 + g for g in range(count)]
    return n.astype(np.int32), m, kinds, seeds


def batch_graph(count: int, seed: int, g: int, log2_n=(8, 18), degree=(4.0, 64.0)):
    """Graph g of graph_batch(count, seed, ...) alone, as (src, dst, n):
    the same sizes, seed and generator, without building the whole batch."""
    n, m, kinds, seeds = batch_params(count, seed, log2_n, degree)
    if kinds[g] == "er":
        src, dst = er(int(n[g]), int(m[g]), seeds[g])
    else:
        src, dst = rmat_graph(int(n[g]), int(m[g]), seeds[g])
    return src, dst, int(n[g])


def graph_batch(count: int, seed: int, log2_n=(8, 18), degree=(4.0, 64.0),
                threads: int = 0, only=None) -> GraphBatch:
    """Generate a batch of `count` graphs (in parallel; deterministic).  With
    `only` (graph indices), just those graphs of the batch, in that order."""
    import concurrent.futures as cf

    n, m, kinds, seeds = batch_params(count, seed, log2_n, degree)
    idx = np.arange(count) if only is None else np.asarray(only, np.int64)
    eo = np.zeros(len(idx) + 1, np.int64)
    eo[1:] = np.cumsum(m[idx])
    src = np.empty(int(eo[-1]), np.int32)
    dst = np.empty(int(eo[-1]), np.int32)
    lib = _load()

    def one(j):
        g = int(idx[j])
        a, b = int(eo[j]), int(eo[j + 1])
        ps = src[a:b].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        pd = dst[a:b].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if kinds[g] == "er":
            rc = lib.gg_er(int(n[g]), b - a, seeds[g], ps, pd)
        else:
            rc = lib.gg_rmat_graph(int(n[g]), b - a, RMAT_ABC[0], RMAT_ABC[1], RMAT_ABC[2],
                                   seeds[g], ps, pd)
        if rc < 0:
            raise ValueError("graph %d (%s, n=%d, m=%d) failed: %d" % (g, kinds[g], n[g], b - a, rc))

    workers = threads or (os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(one, range(len(idx))))
    return GraphBatch(src, dst, eo, n[idx], [kinds[g] for g in idx], [seeds[g] for g in idx])


def rgg_radius(n: int, mean_degree: float = 32.0) -> float:
    """Radius giving the requested mean degree, r = sqrt(d / (pi n))."""
    return math.sqrt(mean_degree / (math.pi * n))


def rgg(n: int, r: float, seed: int):
    """Random geometric graph on n uniform points of the unit square."""
    expect = 0.5 * n * (n - 1) * math.pi * r * r
    cap = int(expect * 1.05 + 6.0 * math.sqrt(expect + 1.0) + 1024)
    while True:
        src = np.empty(cap, np.int32)
        dst = np.empty(cap, np.int32)
        rc = _load().gg_rgg(n, r, seed, _ptr(src), _ptr(dst), cap)
        if rc >= 0:
            return src[:rc].copy(), dst[:rc].copy()
        if rc <= -3:
            cap = -rc - 3
            continue
        raise ValueError("gg_rgg failed: %d" % rc)


def rgg_points(n: int, seed: int):
    """(x, y, perm): the points of rgg(n, r, seed) and the id each one gets."""
    x = np.empty(n, np.float64)
    y = np.empty(n, np.float64)
    perm = np.empty(n, np.int32)
    lib = _load()
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.gg_rgg_point_coords(n, seed, x.ctypes.data_as(f64p), y.ctypes.data_as(f64p))
    lib.gg_rgg_permutation(n, seed, _ptr(perm))
    return x, y, perm


def ba(n: int, k: int, seed: int):
    """Barabasi-Albert: a clique on k + 1 vertices, then each new vertex joins
    k distinct earlier ones drawn in proportion to their degree; permuted ids."""
    m = k * (k + 1) // 2 + (n - k - 1) * k
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gg_ba(n, k, seed, _ptr(src), _ptr(dst))
    if rc != m:
        raise ValueError("gg_ba(n=%d, k=%d) failed: %d" % (n, k, rc))
    return src, dst


def ws(n: int, k: int, p: float, seed: int):
    """Watts-Strogatz: a ring with k neighbours on either side, each edge's far
    end moved with probability p to a vertex outside u's lattice
    neighbourhood; permuted ids; n k pairs (rare coinciding moves repeat)."""
    m = n * k
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gg_ws(n, k, p, seed, _ptr(src), _ptr(dst))
    if rc != m:
        raise ValueError("gg_ws(n=%d, k=%d, p=%g) failed: %d" % (n, k, p, rc))
    return src, dst


# name -> (description, builder)
def _w_er16k():
    return er(16384, 131072, 1001) + (16384,)


def _w_rmat20():
    return rmat(20, 16 * (1 << 20), 1002) + (1 << 20,)


def _w_rgg4m():
    n = 4194304
    return rgg(n, rgg_radius(n), 1003) + (n,)


def _w_rmat24():
    return rmat_distinct(24, 180_000_000, 1004) + (1 << 24,)


def _w_rmat22():
    return rmat_distinct(22, 45_000_000, 1005) + (1 << 22,)


def _w_ba200k():
    return ba(200_000, 50, 1006) + (200_000,)


def _w_ws1m():
    return ws(1_000_000, 25, 0.1, 1007) + (1_000_000,)


WORKLOADS = {
    "er16k": ("Erdos-Renyi G(n=16384, m=131072), seed 1001", _w_er16k),
    "rmat20": ("R-MAT scale 20, 16,777,216 raw draws, permuted ids, seed 1002", _w_rmat20),
    "rgg4m": ("random geometric graph n=4,194,304, r=sqrt(32/(pi n)), seed 1003", _w_rgg4m),
    "rmat24": ("R-MAT scale 24, draws until 180,000,000 distinct edges, seed 1004", _w_rmat24),
    # same density as rmat24 at a quarter of the size: profiling captures
    "rmat22": ("R-MAT scale 22, draws until 45,000,000 distinct edges, seed 1005", _w_rmat22),
    # the paper's two synthetic networks besides the Kronecker graphs, at its
    # sizes (Table 1: 0.2M nodes / 20M directed edges; 1M nodes / 50M)
    "ba200k": ("Barabasi-Albert n=200,000, 50 edges per new vertex, seed 1006", _w_ba200k),
    "ws1m": ("Watts-Strogatz n=1,000,000, 25 neighbours on either side, rewiring "
             "probability 0.1, seed 1007", _w_ws1m),
}


def workload(name: str):
    """Return (src, dst, n) numpy int32 arrays for a named workload."""
    return WORKLOADS[name][1]()
