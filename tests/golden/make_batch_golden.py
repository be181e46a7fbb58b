"""Write tests/golden/batch4096.json: the CPU oracle's triangle count of
every graph of the 4096-graph batched workload.

The workload is graphgen.graph_batch(4096, 1005): half Erdos-Renyi, half
R-MAT (a, b, c = .57, .19, .19), n log-uniform in [2^8, 2^18], mean degree
uniform in [4, 64].  Every stored value comes from ``oracle/`` (the
single-threaded forward algorithm of Sec. II-B) run on ``graphgen``'s seeded
inputs; nothing comes from the GPU library.  The graphs are independent, so
they are counted one graph per host core (a process pool started with
``spawn``).  Usage:

    python tests/golden/make_batch_golden.py [--count 4096] [--workers N]

Stored: the batch parameters, per graph n, the pair count m_in, the number
of distinct undirected edges m, T and the first 16 hex digits of the SHA-256
of its int32 (src, dst) arrays, plus the SHA-256 over all graphs' digests
(pins the generator across hosts) and the oracle's CPU seconds.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch4096.json")
SEED = 1005


def graph_digest(src, dst) -> str:
    import numpy as np

    h = hashlib.sha256()
    h.update(np.ascontiguousarray(src, "<i4").tobytes())
    h.update(np.ascontiguousarray(dst, "<i4").tobytes())
    return h.hexdigest()


def batch_digest(digests) -> str:
    """SHA-256 over the per-graph digests in graph order."""
    h = hashlib.sha256()
    for x in digests:
        h.update(bytes.fromhex(x))
    return h.hexdigest()


def _count_one(job):
    count, g = job
    sys.path.insert(0, ROOT)
    import graphgen
    import oracle

    src, dst, n = graphgen.batch_graph(count, SEED, g)
    t0 = time.process_time()
    r = oracle.forward(src, dst, n, per_vertex=False)
    cpu = time.process_time() - t0
    return g, n, len(src), r["m"], r["T"], graph_digest(src, dst), cpu


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import graphgen
    import oracle

    graphgen.build()
    oracle.build()
    G = args.count
    n_, m_, _, _ = graphgen.batch_params(G, SEED)
    # largest graphs first, so the pool's tail is short
    order = sorted(range(G), key=lambda g: -int(m_[g]))
    rec = [None] * G
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers) as pool:
        done = 0
        for r in pool.imap_unordered(_count_one, [(G, g) for g in order], chunksize=1):
            rec[r[0]] = r
            done += 1
            if done % 256 == 0:
                print("%d/%d graphs, %.0f s" % (done, G, time.time() - t0), flush=True)
    digests = [r[5] for r in rec]
    data = {
        "description": "graphgen.graph_batch(%d, %d): half Erdos-Renyi, half R-MAT "
                       "(.57,.19,.19), n log-uniform in [2^8, 2^18], mean degree uniform in "
                       "[4, 64]; T per graph from the CPU oracle" % (G, SEED),
        "count": G,
        "seed": SEED,
        "log2_n": [8, 18],
        "degree": [4.0, 64.0],
        "batch_sha256": batch_digest(digests),
        "n": [int(r[1]) for r in rec],
        "m_in": [int(r[2]) for r in rec],
        "m": [int(r[3]) for r in rec],
        "T": [int(r[4]) for r in rec],
        "input_sha16": [r[5][:16] for r in rec],
        "oracle_cpu_seconds": round(sum(r[6] for r in rec), 1),
        "wall_seconds": round(time.time() - t0, 1),
        "workers": args.workers,
    }
    with open(OUT, "w") as f:
        json.dump(data, f, separators=(",", ":"))
        f.write("\n")
    print("wrote %s: %d graphs, sum T = %d, %.0f oracle CPU-s" % (
        OUT, G, sum(data["T"]), data["oracle_cpu_seconds"]))


if __name__ == "__main__":
    main()
