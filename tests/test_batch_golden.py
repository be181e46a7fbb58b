"""The stored oracle totals of the 4096-graph batch (tests/golden/batch4096.json)
against the generator and the oracle, on the CPU.

The file is written by tests/golden/make_batch_golden.py from ``oracle/``
alone; here its parameters are checked against graphgen.batch_params, and
the 24 smallest graphs are regenerated (SHA-256 prefix of the pairs) and
recounted by the oracle.  The GPU tests and bench.py compare the library
with these totals.
"""
import hashlib
import json
import os

import numpy as np

import graphgen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096.json")


def load():
    with open(GOLDEN) as f:
        return json.load(f)


def test_parameters_match_the_generator():
    gold = load()
    G = gold["count"]
    assert G == 4096 and gold["seed"] == 1005
    n, m, kinds, _ = graphgen.batch_params(G, gold["seed"])
    assert list(map(int, n)) == gold["n"]
    assert list(map(int, m)) == gold["m_in"]
    for key in ("m", "T", "input_sha16"):
        assert len(gold[key]) == G
    # each graph's pairs are distinct undirected non-loop edges
    assert gold["m"] == gold["m_in"]
    # half Erdos-Renyi (even g), half R-MAT (odd g)
    assert kinds[:4] == ["er", "rmat", "er", "rmat"]
    assert sum(gold["T"]) > 0


def test_smallest_graphs_recounted():
    gold = load()
    G = gold["count"]
    ids = sorted(range(G), key=lambda g: gold["m_in"][g])[:24]
    for g in ids:
        s, d, n = graphgen.batch_graph(G, gold["seed"], g)
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(s, "<i4").tobytes())
        h.update(np.ascontiguousarray(d, "<i4").tobytes())
        assert h.hexdigest()[:16] == gold["input_sha16"][g]
        r = oracle.forward(s, d, n, per_vertex=False)
        assert r["T"] == gold["T"][g] and r["m"] == gold["m"][g]
