"""The 4096-graph batched workload at full size against the CPU oracle.

tests/golden/batch4096.json holds the oracle's triangle count of every graph
of graphgen.graph_batch(4096, 1005) (half Erdos-Renyi, half R-MAT, n
log-uniform in [2^8, 2^18], mean degree uniform in [4, 64]), written by
tests/golden/make_batch_golden.py.  The 64 largest graphs -- the ones whose
unions reach the largest ids, the longest lists and the widest partner
groups -- go through one tc_count_batch call and through two persistent
engines in capacity-sized sub-batches; every total must equal the oracle's
(integer counts: the tolerance is zero).  bench.py compares all 4096.
"""
import concurrent.futures as cf
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096.json")


@pytest.fixture(scope="module")
def tc():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1503_00576_gb300 as lib

    lib.load_library()
    return lib


@pytest.fixture(scope="module")
def largest():
    with open(GOLDEN) as f:
        gold = json.load(f)
    G = gold["count"]
    ids = sorted(range(G), key=lambda g: -gold["m_in"][g])[:64]

    def one(g):
        s, d, n = graphgen.batch_graph(G, gold["seed"], g)
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(s, "<i4").tobytes())
        h.update(np.ascontiguousarray(d, "<i4").tobytes())
        assert h.hexdigest()[:16] == gold["input_sha16"][g], "generator changed (graph %d)" % g
        assert n == gold["n"][g] and len(s) == gold["m_in"][g]
        return s, d, n

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        graphs = list(ex.map(one, ids))
    eo = np.zeros(len(ids) + 1, np.int64)
    eo[1:] = np.cumsum([len(s) for s, _, _ in graphs])
    src = np.concatenate([s for s, _, _ in graphs])
    dst = np.concatenate([d for _, d, _ in graphs])
    vn = np.array([n for _, _, n in graphs], np.int32)
    want = np.array([gold["T"][g] for g in ids], np.uint64)
    return src, dst, eo, vn, want


def test_largest_graphs_in_one_batch(tc, largest):
    import torch

    src, dst, eo, vn, want = largest
    s, d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    got = tc.tc_count_batch(s, d, eo, vn)
    assert np.array_equal(got, want)


def test_largest_graphs_through_engines(tc, largest):
    import torch

    from paper_1503_00576_gb300 import batching

    src, dst, eo, vn, want = largest
    cap = batching.Capacity(pairs=1 << 26, vertices=1 << 22, graphs=64)
    assert len(batching.plan_subbatches(eo, vn, cap)) > 2  # several sub-batches per engine
    s, d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    with batching.BatchCounter(cap) as bc:
        got = bc.count(s, d, eo, vn)
        assert np.array_equal(got, want)
        got = bc.count(src, dst, eo, vn)  # host inputs, copied by the engines
        assert np.array_equal(got, want)
