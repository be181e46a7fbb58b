"""Counting many graphs: sub-batch planning over persistent engines.

A batch engine (tc_engine_*) counts any set of graphs that fits its
capacity in one replay of its captured CUDA graph.  `BatchCounter` splits a
long list of graphs into such sub-batches, in order, and keeps two engines so
that one sub-batch's copy and launch overlap the previous one's run.  A
graph larger than an engine is counted on its own with tc_count.  All
arithmetic happens in the library's kernels; this module only plans and
dispatches.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np

from . import Engine, tc_count, tc_count_host


@dataclass(frozen=True)
class Capacity:
    pairs: int = 1 << 28
    vertices: int = 1 << 25
    graphs: int = 4096


def plan_subbatches(edge_offsets, vertex_counts, cap: Capacity):
    """Greedy, order-preserving split: list of (first, last+1, fits) where
    fits is False for a single graph too large for an engine."""
    eo = np.asarray(edge_offsets, np.int64)
    vn = np.asarray(vertex_counts, np.int64)
    out = []
    g, G = 0, len(vn)
    while g < G:
        pairs = int(eo[g + 1] - eo[g])
        if pairs > cap.pairs or vn[g] > cap.vertices:
            out.append((g, g + 1, False))
            g += 1
            continue
        # extend while the union still fits
        end_p = eo[g] + cap.pairs
        hi = int(np.searchsorted(eo, end_p, side="right")) - 1  # eo[hi] <= end_p
        hi = min(hi, g + cap.graphs, G)
        cv = np.cumsum(vn[g:hi])
        hi = g + int(np.searchsorted(cv, cap.vertices, side="right"))
        hi = max(hi, g + 1)
        out.append((g, hi, True))
        g = hi
    return out


def deal_graphs(edge_offsets, parts: int):
    """Graphs of a batch dealt to `parts` devices: largest first, each to the
    part with the fewest pairs so far (ties: the lower part).  Every graph is
    counted whole on one device, so the parts need no collective; the
    largest graph bounds how even they can be.  Returns one ascending index
    array per part."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    m = np.diff(np.asarray(edge_offsets, np.int64))
    heap = [(0, p) for p in range(parts)]
    out = [[] for _ in range(parts)]
    for g in np.argsort(-m, kind="stable"):
        load, p = heapq.heappop(heap)
        out[p].append(int(g))
        heapq.heappush(heap, (load + int(m[g]), p))
    return [np.array(sorted(x), np.int64) for x in out]


def gather_graphs(src, dst, edge_offsets, vertex_counts, idx):
    """The graphs `idx` of a batch, back to back: (src, dst, edge_offsets,
    vertex_counts) of the smaller batch.  src/dst may be numpy arrays or
    torch tensors (on any device); the pairs are copied, not renumbered
    (ids are local to each graph)."""
    eo = np.asarray(edge_offsets, np.int64)
    vn = np.asarray(vertex_counts, np.int32)
    idx = np.asarray(idx, np.int64)
    spans = [(int(eo[g]), int(eo[g + 1])) for g in idx]
    sub_eo = np.zeros(len(idx) + 1, np.int64)
    sub_eo[1:] = np.cumsum([b - a for a, b in spans])
    if isinstance(src, np.ndarray):
        cat = np.concatenate
        empty = src[:0]
    else:
        import torch

        cat = torch.cat
        empty = src[:0]
    s = cat([src[a:b] for a, b in spans]) if spans else empty
    d = cat([dst[a:b] for a, b in spans]) if spans else dst[:0]
    return s, d, sub_eo, vn[idx]


class BatchCounter:
    """Counts graphs stored back to back (a graphgen.GraphBatch or the same
    three arrays) through two persistent engines."""

    def __init__(self, cap: Capacity = Capacity(), tuning=None, engines: int = 2):
        self.cap = cap
        self.tuning = tuning
        self.engines = [Engine(cap.pairs, cap.vertices, cap.graphs, tuning=tuning)
                        for _ in range(max(1, engines))]

    def close(self):
        for e in self.engines:
            e.close()
        self.engines = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def count(self, src, dst, edge_offsets, vertex_counts) -> np.ndarray:
        """Triangles of every graph.  src/dst: numpy (host) or CUDA tensors
        holding all graphs' pairs back to back."""
        eo = np.asarray(edge_offsets, np.int64)
        vn = np.asarray(vertex_counts, np.int32)
        totals = np.zeros(len(vn), np.uint64)
        plan = plan_subbatches(eo, vn, self.cap)
        on_host = isinstance(src, np.ndarray)
        inflight = []  # (engine, first, last)
        k = 0
        for first, last, fits in plan:
            a, b = int(eo[first]), int(eo[last])
            s, d = src[a:b], dst[a:b]
            if not fits:
                totals[first] = (tc_count_host(s, d, int(vn[first])) if on_host
                                 else tc_count(s, d, int(vn[first])))
                continue
            eng = self.engines[k % len(self.engines)]
            k += 1
            if len(inflight) == len(self.engines):  # engine is busy: collect it first
                e0, f0, l0 = inflight.pop(0)
                totals[f0:l0] = e0.wait()
            eng.submit(s, d, eo[first:last + 1] - a, vn[first:last])
            inflight.append((eng, first, last))
        for e0, f0, l0 in inflight:
            totals[f0:l0] = e0.wait()
        return totals


def count_plain(src, dst, edge_offsets, vertex_counts) -> np.ndarray:
    """The per-graph launch loop the batched path is compared with: one
    tc_count (or tc_count_host) call per graph."""
    eo = np.asarray(edge_offsets, np.int64)
    vn = np.asarray(vertex_counts, np.int32)
    on_host = isinstance(src, np.ndarray)
    out = np.zeros(len(vn), np.uint64)
    for g in range(len(vn)):
        a, b = int(eo[g]), int(eo[g + 1])
        out[g] = (tc_count_host(src[a:b], dst[a:b], int(vn[g])) if on_host
                  else tc_count(src[a:b], dst[a:b], int(vn[g])))
    return out
