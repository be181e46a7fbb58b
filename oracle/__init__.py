"""CPU oracle for exact triangle counting -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The GPU library never imports
it, and it imports nothing from the GPU library.

``forward.c`` is a plain single-threaded C restatement of the sequential
forward algorithm of Polak, arXiv 1503.00576, Sec. II-B (degree order,
forward lists, sorted lists, two-pointer merge per forward edge), plus a
per-vertex count taken straight from the definition of a triangle.  The
derived quantities of the paper's motivation (Sec. I: clustering coefficient
and transitivity ratio) are computed here in float64 from the integer counts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "forward.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

_STATUS = {0: "ok", 1: "invalid argument", 2: "vertex id out of range", 3: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__("oracle: %s (%d)" % (_STATUS.get(code, "?"), code))
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (portable flags, no vector intrinsics)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _bind(lib):
    """Declare the C signatures on a loaded copy of forward.c."""
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.oracle_forward.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int,
                                   u64p, i64p, i32p, i64p, i64p]
    lib.oracle_forward.restype = ctypes.c_int
    lib.oracle_out_degrees.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int, i32p]
    lib.oracle_out_degrees.restype = ctypes.c_int
    lib.oracle_vertex_triangles.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32,
                                            i32p, ctypes.c_int64, i64p]
    lib.oracle_vertex_triangles.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_SO))
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def forward(src, dst, n: int, per_vertex: bool = True, tie_high_first: bool = False) -> dict:
    """Sequential forward algorithm (Sec. II-B).

    Returns ``{"T": int, "t": int64[n] or None, "deg": int32[n], "m": int,
    "max_out_degree": int}``.  Raises OracleError on a bad id or argument.
    """
    s, sp = _i32(src)
    d, dp = _i32(dst)
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    total = ctypes.c_uint64(0)
    m = ctypes.c_int64(0)
    longest = ctypes.c_int64(0)
    deg = np.zeros(max(n, 0), np.int32)
    t = np.zeros(max(n, 0), np.int64) if per_vertex else None
    rc = _load().oracle_forward(
        sp, dp, len(s), n, int(tie_high_first), ctypes.byref(total),
        t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if t is not None else None,
        deg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(m),
        ctypes.byref(longest))
    if rc:
        raise OracleError(rc)
    return {"T": int(total.value), "t": t, "deg": deg, "m": int(m.value),
            "max_out_degree": int(longest.value)}


def out_degrees(src, dst, n: int, tie_high_first: bool = False) -> np.ndarray:
    """|N+(v)| for every v after degree-ordered orientation (Sec. II-B)."""
    s, sp = _i32(src)
    d, dp = _i32(dst)
    out = np.zeros(max(n, 0), np.int32)
    rc = _load().oracle_out_degrees(sp, dp, len(s), n, int(tie_high_first),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc:
        raise OracleError(rc)
    return out


def vertex_triangles(src, dst, n: int, vs) -> np.ndarray:
    """t(v) for the given vertices, from the definition of a triangle."""
    s, sp = _i32(src)
    d, dp = _i32(dst)
    v, vp = _i32(vs)
    out = np.zeros(len(v), np.int64)
    rc = _load().oracle_vertex_triangles(sp, dp, len(s), n, vp, len(v),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc:
        raise OracleError(rc)
    return out


def clustering(t: np.ndarray, deg: np.ndarray) -> np.ndarray:
    """Local clustering coefficient, cc(v) = 2 t(v) / (deg(v) (deg(v) - 1)),
    0 where deg(v) < 2; evaluated in float64 in exactly this order."""
    t = np.asarray(t, np.int64)
    deg = np.asarray(deg, np.int64)
    out = np.zeros(len(t), np.float64)
    ok = deg >= 2
    num = 2.0 * t[ok].astype(np.float64)
    den = deg[ok].astype(np.float64) * (deg[ok] - 1).astype(np.float64)
    out[ok] = num / den
    return out


def transitivity(T: int, deg: np.ndarray) -> float:
    """Transitivity ratio 3T / (number of paths of length two), 0 if none.
    Both integers are exact; one float64 division."""
    deg = np.asarray(deg, np.int64)
    wedges = int((deg * (deg - 1) // 2).sum())
    if wedges == 0:
        return 0.0
    return float(np.float64(3 * T) / np.float64(wedges))
