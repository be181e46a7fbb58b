"""Write tests/golden/workloads.json from the CPU oracle.

Every stored value comes from ``oracle/`` run on the seeded inputs of
``graphgen`` (nothing from the GPU library).  Usage:

    python tests/golden/make_golden.py [workload ...]

Stored per workload: the SHA-256 of the generated int32 (src, dst) arrays
(pins the generator across hosts), n, the input pair count m_in, the
number of distinct undirected edges m, the triangle count T, the longest
forward list, the SHA-256 of the per-vertex counts t (int64, little-endian)
and of the degrees (int32), the transitivity ratio, and t(v) for a fixed
sample of vertices (the highest-degree ones plus seeded random ones), each
cross-checked with the definition-based per-vertex count.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")


def input_sha(src, dst) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(src, "<i4").tobytes())
    h.update(np.ascontiguousarray(dst, "<i4").tobytes())
    return h.hexdigest()


def array_sha(a, dtype) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype).tobytes()).hexdigest()


def sample_vertices(deg: np.ndarray, seed: int, k_top: int = 4, k_rand: int = 12) -> np.ndarray:
    top = np.argsort(-deg.astype(np.int64), kind="stable")[:k_top]
    rng = np.random.default_rng(seed)
    rnd = rng.choice(len(deg), size=k_rand, replace=False)
    return np.unique(np.concatenate([top, rnd])).astype(np.int32)


def make(name: str) -> dict:
    t0 = time.time()
    src, dst, n = graphgen.workload(name)
    t1 = time.time()
    r = oracle.forward(src, dst, n)
    t2 = time.time()
    vs = sample_vertices(r["deg"], 7 + len(name))
    direct = oracle.vertex_triangles(src, dst, n, vs)
    if not np.array_equal(direct, r["t"][vs]):
        raise SystemExit("definition-based t(v) disagrees with the forward oracle on " + name)
    if int(r["t"].sum()) != 3 * r["T"]:
        raise SystemExit("sum of t != 3T on " + name)
    rec = {
        "description": graphgen.WORKLOADS[name][0],
        "input_sha256": input_sha(src, dst),
        "n": int(n),
        "m_in": int(len(src)),
        "m": r["m"],
        "T": r["T"],
        "max_out_degree": r["max_out_degree"],
        "max_degree": int(r["deg"].max()),
        "t_sha256": array_sha(r["t"], "<i8"),
        "deg_sha256": array_sha(r["deg"], "<i4"),
        "transitivity": oracle.transitivity(r["T"], r["deg"]),
        "sample_vertices": [int(v) for v in vs],
        "sample_t": [int(x) for x in r["t"][vs]],
        "sample_deg": [int(x) for x in r["deg"][vs]],
        "oracle_seconds": round(t2 - t1, 1),
        "generate_seconds": round(t1 - t0, 1),
    }
    return rec


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        print("workload", name, flush=True)
        data[name] = make(name)
        print(json.dumps(data[name], indent=1), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or list(graphgen.WORKLOADS))
