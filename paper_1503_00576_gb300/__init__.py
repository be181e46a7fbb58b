"""Exact triangle counting on GB300 (sm_103a): Python binding of libtc.

The forward algorithm of A. Polak, "Counting Triangles in Large Graphs on
GPU" (arXiv 1503.00576): every step runs in the CUDA kernels of libtc.so
behind the C ABI of ``include/tc.h``; this module only marshals arguments
(torch tensors for device memory and streams, numpy arrays for host
buffers).  There is no CPU fallback: if the library is missing or no GPU is
present, calls raise.

Functions mirror the C ABI names:

    tc_count(src, dst, n)                  -> T
    tc_count_per_vertex(src, dst, n)       -> (T, t int64[n], deg int32[n])
    tc_clustering(t, deg)                  -> (cc float64[n], transitivity)
    tc_count_host(src, dst, n)             -> T          (host arrays in, transfers inside)
    tc_count_per_vertex_host(src, dst, n)  -> (T, t, deg) (numpy in and out)
    tc_workspace_bytes(m, n), tc_count_ws(src, dst, n, ws)
    tc_count_batch(src, dst, edge_offsets, vertex_counts) -> uint64[G]
    Engine(max_pairs, max_vertices, max_graphs).count(...)  (tc_engine_*)
    tc_set_tuning(dict), tc_get_tuning()
    tc_count_noalloc(src, dst, n)
    tc_launch_count(), tc_profile_enable(on), tc_profile_read(reset)

``src`` / ``dst`` are int32 CUDA tensors of the same length (pair i is the
undirected edge {src[i], dst[i]}); ``n`` is the vertex count.

Environment: ``TC_TUNING``, a JSON object of tc_tuning fields (for example
``{"heavy_ratio_pct": 150}``), sets the process-wide tuning when the library
is loaded; a value the library refuses raises TCError there.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtc.so")

TC_OK = 0
TC_ERR_INVALID_ARG = 1
TC_ERR_ID_RANGE = 2
TC_ERR_OOM = 3
TC_ERR_CUDA = 4
TC_ERR_TIMEOUT = 5
TC_ERR_OVERFLOW = 6
TC_COUNT_ERROR = (1 << 64) - 1
PHASES = ("canon", "rank", "orient", "sort", "offsets", "lists", "groups", "count")

# Every symbol include/tc.h and include/tc_debug.h declare.
EXPORTS = ("tc_count", "tc_count_per_vertex", "tc_count_part", "tc_count_per_vertex_part",
           "tc_clustering", "tc_count_host",
           "tc_count_per_vertex_host", "tc_workspace_bytes", "tc_count_ws", "tc_set_tuning",
           "tc_get_tuning", "tc_count_batch", "tc_engine_create", "tc_engine_submit",
           "tc_engine_wait", "tc_engine_submit_parts", "tc_engine_poll", "tc_engine_count",
           "tc_engine_destroy", "tc_count_work", "tc_count_work_part", "tc_count_noalloc",
           "tc_last_error", "tc_status_string", "tc_last_error_detail", "tc_launch_count",
           "tc_profile_enable", "tc_profile_read", "tc_phase_name",
           "tc_debug_set_wait_limit", "tc_debug_fail_allocations", "tc_debug_reset")


class Work(ctypes.Structure):
    """tc_work: what the counting phase does for one graph."""
    _fields_ = [("edges", ctypes.c_int64), ("lookups", ctypes.c_int64),
                ("inserts", ctypes.c_int64), ("merge_work", ctypes.c_int64),
                ("triangles", ctypes.c_uint64), ("max_out_degree", ctypes.c_int32),
                ("vertices", ctypes.c_int32), ("hub_lookups", ctypes.c_int64 * 4),
                ("dense_triangles", ctypes.c_uint64), ("dense_vertices", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    """tc_tuning: how partner groups map onto warps/CTAs and which list is hashed."""
    _fields_ = [("warp_max_list", ctypes.c_int32), ("warp_max_partners", ctypes.c_int32),
                ("heavy_ratio_pct", ctypes.c_int32), ("hub_min_edges", ctypes.c_int64),
                ("hub_vertices", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


DEFAULT_TUNING = {"warp_max_list": 128, "warp_max_partners": 64, "heavy_ratio_pct": 100,
                  "hub_min_edges": 1 << 21, "hub_vertices": 1 << 14}


class TCError(RuntimeError):
    """A libtc call returned an error status."""

    def __init__(self, code: int, detail: str):
        super().__init__("libtc: %s (%d)%s" % (_status_name(code), code,
                                              ": " + detail if detail else ""))
        self.code = code
        self.detail = detail


_lib = None
_lock = threading.Lock()


def _bind(lib):
    c = ctypes
    vp, i64, i32, u64, sz = c.c_void_p, c.c_int64, c.c_int32, c.c_uint64, c.c_size_t
    sig = {
        "tc_count": ([vp, vp, i64, i32, vp], u64),
        "tc_count_per_vertex": ([vp, vp, i64, i32, vp, vp, vp, c.POINTER(u64)], c.c_int),
        "tc_count_part": ([vp, vp, i64, i32, i32, i32, vp, c.POINTER(u64)], c.c_int),
        "tc_count_per_vertex_part": ([vp, vp, i64, i32, i32, i32, vp, vp, vp, c.POINTER(u64)],
                                     c.c_int),
        "tc_clustering": ([vp, vp, i32, vp, vp, c.POINTER(c.c_double)], c.c_int),
        "tc_count_host": ([vp, vp, i64, i32, c.POINTER(u64)], c.c_int),
        "tc_count_per_vertex_host": ([vp, vp, i64, i32, vp, vp, c.POINTER(u64)], c.c_int),
        "tc_workspace_bytes": ([i64, i32], sz),
        "tc_count_ws": ([vp, vp, i64, i32, vp, vp, sz, c.POINTER(u64)], c.c_int),
        "tc_count_noalloc": ([vp, vp, i64, i32, vp, c.POINTER(u64)], c.c_int),
        "tc_count_work": ([vp, vp, i64, i32, vp, vp], c.c_int),
        "tc_count_work_part": ([vp, vp, i64, i32, i32, i32, vp, vp], c.c_int),
        "tc_set_tuning": ([c.POINTER(Tuning)], c.c_int),
        "tc_get_tuning": ([c.POINTER(Tuning)], c.c_int),
        "tc_count_batch": ([vp, vp, i32, vp, vp, vp, vp], c.c_int),
        "tc_engine_create": ([i64, i32, i32, c.POINTER(Tuning), c.POINTER(vp)], c.c_int),
        "tc_engine_submit": ([vp, vp, vp, i32, i32, vp, vp], c.c_int),
        "tc_engine_wait": ([vp, vp], c.c_int),
        "tc_engine_submit_parts": ([vp, i32, vp, vp, vp, vp, i32], c.c_int),
        "tc_engine_poll": ([vp], i32),
        "tc_engine_count": ([vp, vp, vp, i32, i32, vp, vp, vp], c.c_int),
        "tc_engine_destroy": ([vp], c.c_int),
        "tc_last_error": ([], c.c_int),
        "tc_status_string": ([c.c_int], c.c_char_p),
        "tc_last_error_detail": ([], c.c_char_p),
        "tc_launch_count": ([], u64),
        "tc_profile_enable": ([c.c_int], None),
        "tc_profile_read": ([c.POINTER(c.c_double), c.POINTER(u64), c.c_int], None),
        "tc_phase_name": ([c.c_int], c.c_char_p),
        "tc_debug_set_wait_limit": ([c.c_uint32, i32], c.c_int),
        "tc_debug_fail_allocations": ([i32, i32], c.c_int),
        "tc_debug_reset": ([], c.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def load_library(path: str = LIB_PATH):
    """Load libtc.so (build it with ``python -m paper_1503_00576_gb300.build``)."""
    global _lib
    fresh = False
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    "libtc.so not found at %s: build it with "
                    "`python -m paper_1503_00576_gb300.build` (nvcc, sm_103a). "
                    "There is no CPU fallback." % path)
            _lib = _bind(ctypes.CDLL(path))
            fresh = True
    if fresh and os.environ.get("TC_TUNING"):
        tc_set_tuning(json.loads(os.environ["TC_TUNING"]))
    return _lib


def _status_name(code: int) -> str:
    names = {0: "ok", 1: "invalid argument", 2: "vertex id out of range", 3: "out of device memory",
             4: "CUDA error", 5: "device wait timed out", 6: "size beyond limits"}
    return names.get(code, "unknown status")


def _check(code: int):
    if code != TC_OK:
        raise TCError(code, load_library().tc_last_error_detail().decode())


def _check_batch(code: int, totals: np.ndarray):
    """Batch calls: TC_ERR_ID_RANGE fails only the graphs that hold a bad id
    (their totals are TC_COUNT_ERROR); the error carries every total."""
    if code != TC_OK:
        err = TCError(code, load_library().tc_last_error_detail().decode())
        if code == TC_ERR_ID_RANGE:
            err.totals = totals
        raise err


def _torch():
    import torch

    return torch


def _stream_of(stream, device):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _edges(src, dst):
    torch = _torch()
    for name, x in (("src", src), ("dst", dst)):
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if x.dtype != torch.int32:
            raise TypeError("%s must be int32, got %s" % (name, x.dtype))
        if x.dim() != 1 or not x.is_contiguous():
            raise TypeError("%s must be 1-D and contiguous" % name)
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    if src.device != dst.device:
        raise ValueError("src and dst are on different devices")
    return src.device


def tc_count(src, dst, n: int, stream=None) -> int:
    """Triangle count T (uint64) of the graph given by the pairs (src[i], dst[i])."""
    torch = _torch()
    dev = _edges(src, dst)
    lib = load_library()
    with torch.cuda.device(dev):
        T = lib.tc_count(src.data_ptr(), dst.data_ptr(), src.numel(), n, _stream_of(stream, dev))
    if T == TC_COUNT_ERROR:
        _check(lib.tc_last_error())
    return int(T)


def tc_count_per_vertex(src, dst, n: int, stream=None, t_out=None, deg_out=None):
    """(T, t, deg): t[v] = triangles containing v (int64), deg[v] = degree of
    v in the simple graph (int32), both device tensors of length n."""
    torch = _torch()
    dev = _edges(src, dst)
    t = t_out if t_out is not None else torch.empty(n, dtype=torch.int64, device=dev)
    deg = deg_out if deg_out is not None else torch.empty(n, dtype=torch.int32, device=dev)
    if t.dtype != torch.int64 or t.numel() != n or deg.dtype != torch.int32 or deg.numel() != n:
        raise TypeError("t_out must be int64[n] and deg_out int32[n]")
    total = ctypes.c_uint64(0)
    lib = load_library()
    with torch.cuda.device(dev):
        rc = lib.tc_count_per_vertex(src.data_ptr(), dst.data_ptr(), src.numel(), n,
                                     _stream_of(stream, dev), t.data_ptr(), deg.data_ptr(),
                                     ctypes.byref(total))
    _check(rc)
    return int(total.value), t, deg


def tc_count_part(src, dst, n: int, part: int, parts: int, stream=None) -> int:
    """This part's share of T when the counting is split into `parts`
    shares (the shares of parts 0 .. parts-1 add up to T)."""
    torch = _torch()
    dev = _edges(src, dst)
    total = ctypes.c_uint64(0)
    lib = load_library()
    with torch.cuda.device(dev):
        rc = lib.tc_count_part(src.data_ptr(), dst.data_ptr(), src.numel(), n, part, parts,
                               _stream_of(stream, dev), ctypes.byref(total))
    _check(rc)
    return int(total.value)


def tc_count_per_vertex_part(src, dst, n: int, part: int, parts: int, stream=None,
                             t_out=None, deg_out=None):
    """(T_part, t_part, deg): this part's shares of T and of t (they add up
    over the parts to T and t) and the complete degrees."""
    torch = _torch()
    dev = _edges(src, dst)
    t = t_out if t_out is not None else torch.empty(n, dtype=torch.int64, device=dev)
    deg = deg_out if deg_out is not None else torch.empty(n, dtype=torch.int32, device=dev)
    if t.dtype != torch.int64 or t.numel() != n or deg.dtype != torch.int32 or deg.numel() != n:
        raise TypeError("t_out must be int64[n] and deg_out int32[n]")
    total = ctypes.c_uint64(0)
    lib = load_library()
    with torch.cuda.device(dev):
        rc = lib.tc_count_per_vertex_part(src.data_ptr(), dst.data_ptr(), src.numel(), n, part,
                                          parts, _stream_of(stream, dev), t.data_ptr(),
                                          deg.data_ptr(), ctypes.byref(total))
    _check(rc)
    return int(total.value), t, deg


def tc_clustering(t, deg, stream=None, want_cc: bool = True):
    """(cc, transitivity): local clustering coefficients (float64 device
    tensor, or None) and the transitivity ratio (float)."""
    torch = _torch()
    if t.dtype != torch.int64 or deg.dtype != torch.int32 or t.numel() != deg.numel():
        raise TypeError("t must be int64[n] and deg int32[n]")
    n = t.numel()
    cc = torch.empty(n, dtype=torch.float64, device=t.device) if want_cc else None
    tr = ctypes.c_double(0.0)
    lib = load_library()
    with torch.cuda.device(t.device):
        rc = lib.tc_clustering(t.data_ptr(), deg.data_ptr(), n, _stream_of(stream, t.device),
                               cc.data_ptr() if cc is not None else None, ctypes.byref(tr))
    _check(rc)
    return cc, float(tr.value)


def _host_i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a


def tc_count_host(src, dst, n: int) -> int:
    """T from HOST arrays (numpy int32 or pinned CPU tensors); the transfers
    to and from the device are part of the call (where the device reads host
    memory through the host's page tables, the inputs are read in place)."""
    s, d = _host_ptrs(src, dst)
    total = ctypes.c_uint64(0)
    _check(load_library().tc_count_host(s[1], d[1], s[2], n, ctypes.byref(total)))
    return int(total.value)


def tc_count_per_vertex_host(src, dst, n: int, t_out=None, deg_out=None):
    """(T, t, deg) from and into HOST buffers (numpy arrays or CPU tensors)."""
    s, d = _host_ptrs(src, dst)
    t = t_out if t_out is not None else np.empty(n, np.int64)
    deg = deg_out if deg_out is not None else np.empty(n, np.int32)
    total = ctypes.c_uint64(0)
    _check(load_library().tc_count_per_vertex_host(s[1], d[1], s[2], n, _host_ptr(t, 8),
                                                   _host_ptr(deg, 4), ctypes.byref(total)))
    return int(total.value), t, deg


def _host_ptr(x, itemsize):
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous or x.itemsize != itemsize:
            raise TypeError("host buffer must be contiguous with %d-byte items" % itemsize)
        return x.ctypes.data
    torch = _torch()
    if isinstance(x, torch.Tensor) and not x.is_cuda and x.is_contiguous() \
            and x.element_size() == itemsize:
        return x.data_ptr()
    raise TypeError("expected a numpy array or a contiguous CPU tensor")


def _host_ptrs(src, dst):
    out = []
    for x in (src, dst):
        if isinstance(x, np.ndarray):
            if x.dtype != np.int32 or not x.flags.c_contiguous:
                raise TypeError("host edge arrays must be contiguous int32")
            out.append((x, x.ctypes.data, len(x)))
        else:
            torch = _torch()
            if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != torch.int32 \
                    or not x.is_contiguous():
                raise TypeError("host edge arrays must be contiguous int32 CPU tensors")
            out.append((x, x.data_ptr(), x.numel()))
    if out[0][2] != out[1][2]:
        raise ValueError("src and dst differ in length")
    return out


def tc_workspace_bytes(m: int, n: int) -> int:
    return int(load_library().tc_workspace_bytes(m, n))


def tc_count_ws(src, dst, n: int, ws, stream=None) -> int:
    """T using the caller's workspace ``ws`` (a CUDA uint8 tensor of at least
    tc_workspace_bytes(m, n) bytes); libtc allocates nothing."""
    torch = _torch()
    dev = _edges(src, dst)
    total = ctypes.c_uint64(0)
    lib = load_library()
    with torch.cuda.device(dev):
        rc = lib.tc_count_ws(src.data_ptr(), dst.data_ptr(), src.numel(), n,
                             _stream_of(stream, dev), ws.data_ptr(),
                             ws.numel() * ws.element_size(), ctypes.byref(total))
    _check(rc)
    return int(total.value)


def tc_set_tuning(tuning=None) -> None:
    """Process-wide tuning for subsequent calls (None restores the defaults)."""
    if tuning is None:
        _check(load_library().tc_set_tuning(None))
        return
    t = Tuning(**{**DEFAULT_TUNING, **dict(tuning)})
    _check(load_library().tc_set_tuning(ctypes.byref(t)))


def tc_get_tuning() -> dict:
    t = Tuning()
    _check(load_library().tc_get_tuning(ctypes.byref(t)))
    return t.as_dict()


def _batch_arrays(edge_offsets, vertex_counts):
    eo = np.ascontiguousarray(edge_offsets, dtype=np.int64)
    vn = np.ascontiguousarray(vertex_counts, dtype=np.int32)
    if eo.ndim != 1 or vn.ndim != 1 or len(eo) != len(vn) + 1:
        raise ValueError("edge_offsets must have one entry more than vertex_counts")
    return eo, vn


def tc_count_batch(src, dst, edge_offsets, vertex_counts, stream=None) -> np.ndarray:
    """Triangles of each graph of a batch (uint64[G]).

    ``src``/``dst``: int32 CUDA tensors holding every graph's pairs back to
    back, graph g at [edge_offsets[g], edge_offsets[g+1]) with ids local to
    the graph (< vertex_counts[g]).  The batch is counted as one disjoint
    union in a single pass.  A graph with an id out of range fails alone:
    TCError(TC_ERR_ID_RANGE) whose ``totals`` hold TC_COUNT_ERROR for it and
    the exact count of every other graph."""
    torch = _torch()
    dev = _edges(src, dst)
    eo, vn = _batch_arrays(edge_offsets, vertex_counts)
    if eo[-1] > src.numel():
        raise ValueError("edge_offsets run past the edge arrays")
    out = np.zeros(len(vn), np.uint64)
    lib = load_library()
    with torch.cuda.device(dev):
        rc = lib.tc_count_batch(src.data_ptr(), dst.data_ptr(), len(vn), eo.ctypes.data,
                                vn.ctypes.data, _stream_of(stream, dev), out.ctypes.data)
    _check_batch(rc, out)
    return out


class Engine:
    """Persistent batch engine (tc_engine_*): fixed device buffers and a
    CUDA graph of the whole batch pipeline, replayed for every batch.

    ``submit`` returns immediately (the batch runs on the engine's stream);
    ``wait`` returns the per-graph counts.  Host inputs must stay alive (and
    unmodified) until ``wait``; page-locked ones overlap best."""

    def __init__(self, max_pairs: int, max_vertices: int, max_graphs: int, tuning=None,
                 device=None):
        torch = _torch()
        self.lib = load_library()
        self.max_pairs, self.max_vertices, self.max_graphs = max_pairs, max_vertices, max_graphs
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.tuning = {**DEFAULT_TUNING, **(dict(tuning) if tuning else {})}
        t = Tuning(**self.tuning)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.tc_engine_create(max_pairs, max_vertices, max_graphs, ctypes.byref(t),
                                           ctypes.byref(h))
        _check(rc)
        self._h = h
        self._pending = None

    def submit(self, src, dst, edge_offsets, vertex_counts) -> None:
        torch = _torch()
        eo, vn = _batch_arrays(edge_offsets, vertex_counts)
        if isinstance(src, np.ndarray):
            s = np.ascontiguousarray(src, np.int32)
            d = np.ascontiguousarray(dst, np.int32)
            ps, pd, on_host = s.ctypes.data, d.ctypes.data, 1
            keep = (s, d)
        elif isinstance(src, torch.Tensor) and not src.is_cuda:
            s, d = src.contiguous(), dst.contiguous()
            if s.dtype != torch.int32 or d.dtype != torch.int32:
                raise TypeError("edge arrays must be int32")
            ps, pd, on_host = s.data_ptr(), d.data_ptr(), 1
            keep = (s, d)
        else:
            _edges(src, dst)
            ps, pd, on_host = src.data_ptr(), dst.data_ptr(), 0
            keep = (src, dst)
        if eo[-1] > (len(keep[0]) if on_host else keep[0].numel()):
            raise ValueError("edge_offsets run past the edge arrays")
        with torch.cuda.device(self.device):
            rc = self.lib.tc_engine_submit(self._h, ps, pd, on_host, len(vn), eo.ctypes.data,
                                           vn.ctypes.data)
        _check(rc)
        self._pending = (keep, eo, vn)

    def submit_parts(self, graphs, on_host: bool) -> None:
        """graphs: list of (src, dst, n), each a pair of int32 arrays (numpy
        or pinned CPU tensors when on_host, CUDA tensors otherwise)."""
        torch = _torch()
        G = len(graphs)
        ps = (ctypes.c_void_p * max(G, 1))()
        pd = (ctypes.c_void_p * max(G, 1))()
        pc = np.zeros(max(G, 1), np.int64)
        vn = np.zeros(max(G, 1), np.int32)
        keep = []
        for i, (s, d, n) in enumerate(graphs):
            if isinstance(s, np.ndarray):
                s = np.ascontiguousarray(s, np.int32)
                d = np.ascontiguousarray(d, np.int32)
                ps[i], pd[i], cnt = s.ctypes.data, d.ctypes.data, len(s)
            else:
                ps[i], pd[i], cnt = s.data_ptr(), d.data_ptr(), s.numel()
            pc[i], vn[i] = cnt, n
            keep.append((s, d))
        with torch.cuda.device(self.device):
            rc = self.lib.tc_engine_submit_parts(self._h, G, ps, pd, pc.ctypes.data,
                                                 vn.ctypes.data, 1 if on_host else 0)
        _check(rc)
        self._pending = (keep, None, vn[:G])

    def poll(self) -> bool:
        """True when no batch is running (wait() will not block)."""
        return bool(self.lib.tc_engine_poll(self._h))

    def wait(self) -> np.ndarray:
        if self._pending is None:
            raise RuntimeError("no batch submitted")
        n = len(self._pending[2])
        out = np.zeros(n, np.uint64)
        rc = self.lib.tc_engine_wait(self._h, out.ctypes.data)
        self._pending = None
        _check_batch(rc, out)
        return out

    def count(self, src, dst, edge_offsets, vertex_counts) -> np.ndarray:
        self.submit(src, dst, edge_offsets, vertex_counts)
        return self.wait()

    def close(self) -> None:
        if getattr(self, "_h", None):
            self.lib.tc_engine_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tc_count_work(src, dst, n: int, stream=None, part: int = 0, parts: int = 1) -> dict:
    """Work of the counting phase for this graph (tc_work as a dict): hash
    lookups and inserts, the merge work W of a sorted-list merge, the largest
    out-degree, m and T; with parts > 1, the work of share `part`
    (tc_count_work_part).  Instrumentation: runs the whole pipeline once."""
    torch = _torch()
    dev = _edges(src, dst)
    w = Work()
    lib = load_library()
    with torch.cuda.device(dev):
        rc = lib.tc_count_work_part(src.data_ptr(), dst.data_ptr(), src.numel(), n, part, parts,
                                    _stream_of(stream, dev), ctypes.byref(w))
    _check(rc)
    out = {f: int(getattr(w, f)) for f, _ in w._fields_ if f not in ("hub_lookups", "pad_")}
    out["hub_lookups"] = {1 << (12 + i): int(w.hub_lookups[i]) for i in range(4)}
    return out


TC_NOALLOC_SCRATCH_BYTES = 32 << 20


def tc_count_noalloc(src, dst, n: int, stream=None) -> int:
    """T without any allocation inside the library: for callers that cannot
    allocate device memory while they run.  Scratch is a static device array
    of TC_NOALLOC_SCRATCH_BYTES shared by all calls, so calls must not
    overlap on the GPU; graphs needing more scratch raise TCError
    (TC_ERR_OVERFLOW)."""
    torch = _torch()
    dev = _edges(src, dst)
    total = ctypes.c_uint64(0)
    lib = load_library()
    with torch.cuda.device(dev):
        rc = lib.tc_count_noalloc(src.data_ptr(), dst.data_ptr(), src.numel(), n,
                                  _stream_of(stream, dev), ctypes.byref(total))
    _check(rc)
    return int(total.value)


def tc_launch_count() -> int:
    return int(load_library().tc_launch_count())


def tc_profile_enable(on: bool = True) -> None:
    load_library().tc_profile_enable(1 if on else 0)


def tc_profile_read(reset: bool = False) -> dict:
    """{phase: (ms, launches)} accumulated since the last reset."""
    ms = (ctypes.c_double * len(PHASES))()
    nl = (ctypes.c_uint64 * len(PHASES))()
    load_library().tc_profile_read(ms, nl, 1 if reset else 0)
    return {p: (float(ms[i]), int(nl[i])) for i, p in enumerate(PHASES)}


def tc_debug_set_wait_limit(spin_limit: int, unpublished_tile: int = -1, device=None) -> None:
    """Failure-path test hook (include/tc_debug.h): every device spin-wait on
    `device` gives up after `spin_limit` iterations, and radix-sort tile
    `unpublished_tile` (>= 0) never publishes, so the tiles after it wait on
    a word nothing sets.  Calls then fail with TC_ERR_TIMEOUT."""
    torch = _torch()
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        _check(load_library().tc_debug_set_wait_limit(spin_limit, unpublished_tile))


def tc_debug_fail_allocations(skip: int, count: int) -> None:
    """Failure-path test hook: of the library's next device allocations the
    first `skip` succeed and the `count` after them fail (TC_ERR_OOM)."""
    _check(load_library().tc_debug_fail_allocations(skip, count))


def tc_debug_reset(device=None) -> None:
    """Undo both failure-path hooks (wait limit on `device`)."""
    torch = _torch()
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        _check(load_library().tc_debug_reset())


# short aliases
count = tc_count
count_per_vertex = tc_count_per_vertex
clustering = tc_clustering
