"""Autotuner for the counting layout (tc_tuning).

The knobs decide how partner groups map onto the GPU -- one warp or a whole
CTA per group (list-length and partner-count thresholds) -- and which list
of an edge is hashed (the degree-ratio switch).  Counts never depend on
them; speed does, and the best setting depends on the graphs' size and
degree mix.  `tune_batches` times each candidate on a sample sub-batch of the
workload with a fresh engine; `tune_graph` does the same for single-graph
calls (process-wide tuning).  Results are cached in a JSON file keyed by the
device and a coarse description of the workload.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import DEFAULT_TUNING, Engine, _torch, tc_count, tc_set_tuning
from .batching import Capacity, plan_subbatches

CANDIDATES = [{**DEFAULT_TUNING, **c} for c in (
    {},
    {"warp_max_list": 64, "warp_max_partners": 32, "heavy_ratio_pct": 100},
    {"warp_max_list": 128, "warp_max_partners": 128, "heavy_ratio_pct": 100},
    {"warp_max_list": 32, "warp_max_partners": 16, "heavy_ratio_pct": 100},
    {"warp_max_list": 128, "warp_max_partners": 64, "heavy_ratio_pct": 150},
    {"warp_max_list": 128, "warp_max_partners": 64, "heavy_ratio_pct": 300},
)]

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning_cache_v2.json")


def _device_key() -> str:
    torch = _torch()
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%dsm" % (p.name, p.multi_processor_count)


def workload_key(edge_offsets, vertex_counts) -> str:
    """Coarse shape: graphs, log2 of median edges and of mean degree."""
    eo = np.asarray(edge_offsets, np.int64)
    vn = np.asarray(vertex_counts, np.int64)
    m = np.diff(eo)
    med = int(np.log2(max(1, int(np.median(m))))) if len(m) else 0
    deg = int(np.log2(max(1.0, 2.0 * m.sum() / max(1, vn.sum()))))
    return "g%d/m2^%d/d2^%d" % (min(len(vn), 4096), med, deg)


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, rec: dict) -> None:
    data = _load_cache()
    data[key] = rec
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune_batches(src, dst, edge_offsets, vertex_counts, cap: Capacity = Capacity(),
                 candidates=None, repeats: int = 2, use_cache: bool = True) -> dict:
    """Best tuning for counting these graphs in sub-batches of `cap`.

    Times every candidate on the first sub-batch (the plan's largest
    typical unit of work) with its own engine; returns
    {"tuning": {...}, "ms": {...}, "key": str, "cached": bool}."""
    torch = _torch()
    key = "batch/%s/%s/p%d" % (_device_key(), workload_key(edge_offsets, vertex_counts),
                               cap.pairs)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return {**hit, "key": key, "cached": True}
    eo = np.asarray(edge_offsets, np.int64)
    vn = np.asarray(vertex_counts, np.int32)
    first, last, _ = next(p for p in plan_subbatches(eo, vn, cap) if p[2])
    a, b = int(eo[first]), int(eo[last])
    s, d = src[a:b], dst[a:b]
    seo, svn = eo[first:last + 1] - a, vn[first:last]
    ms = {}
    for cand in candidates or CANDIDATES:
        with Engine(cap.pairs, cap.vertices, cap.graphs, tuning=cand) as eng:
            ref = eng.count(s, d, seo, svn)  # warm
            times = []
            for _ in range(repeats):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                got = eng.count(s, d, seo, svn)
                times.append(time.perf_counter() - t0)
                if not np.array_equal(got, ref):
                    raise RuntimeError("tuning changed a count: %r" % (cand,))
        ms[json.dumps(cand, sort_keys=True)] = 1e3 * min(times)
    best = min(ms, key=ms.get)
    rec = {"tuning": json.loads(best), "ms": ms, "sample_graphs": last - first,
           "sample_pairs": b - a}
    _store(key, rec)
    return {**rec, "key": key, "cached": False}


def tune_graph(src, dst, n: int, candidates=None, repeats: int = 2,
               use_cache: bool = True) -> dict:
    """Best process-wide tuning for single-graph calls on graphs like this
    one; leaves it set (tc_set_tuning) and returns the record."""
    torch = _torch()
    m = int(src.numel())
    key = "graph/%s/m2^%d/d2^%d" % (_device_key(), int(np.log2(max(1, m))),
                                    int(np.log2(max(1.0, 2.0 * m / max(1, n)))))
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            tc_set_tuning(hit["tuning"])
            return {**hit, "key": key, "cached": True}
    ms = {}
    ref = None
    for cand in candidates or CANDIDATES:
        tc_set_tuning(cand)
        got = tc_count(src, dst, n)
        ref = got if ref is None else ref
        if got != ref:
            raise RuntimeError("tuning changed the count: %r" % (cand,))
        times = []
        for _ in range(repeats):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tc_count(src, dst, n)
            times.append(time.perf_counter() - t0)
        ms[json.dumps(cand, sort_keys=True)] = 1e3 * min(times)
    best = json.loads(min(ms, key=ms.get))
    tc_set_tuning(best)
    rec = {"tuning": best, "ms": ms}
    _store(key, rec)
    return {**rec, "key": key, "cached": False}
