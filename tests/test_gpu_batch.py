"""Batched counting: every graph of a batch gets exactly its count alone.

A batch is counted as the disjoint union of its graphs.  The checks:
per-graph totals against the CPU oracle, against single-graph tc_count, the
persistent CUDA-graph engine against both (host and device inputs, batches
of changing size), invariance under every tuning, and the error paths.
Integer counts: the tolerance is zero.
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1503_00576_gb300 as lib

    lib.load_library()
    return lib


@pytest.fixture(scope="module")
def batch():
    return graphgen.graph_batch(48, 11, log2_n=(5, 12), degree=(2.0, 40.0))


@pytest.fixture(scope="module")
def expected(batch):
    return np.array([oracle.forward(*batch.graph(g), per_vertex=False)["T"]
                     for g in range(len(batch))], np.uint64)


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def test_batch_matches_oracle(tc, batch, expected):
    got = tc.tc_count_batch(dev(batch.src), dev(batch.dst), batch.edge_offsets,
                            batch.vertex_counts)
    assert np.array_equal(got, expected)
    assert expected.sum() > 0


def test_alone_equals_in_batch(tc, batch, expected):
    for g in range(0, len(batch), 5):
        s, d, n = batch.graph(g)
        assert tc.tc_count(dev(s), dev(d), n) == expected[g]


def test_engine_host_and_device_inputs(tc, batch, expected):
    with tc.Engine(int(batch.edge_offsets[-1]) + 1000, int(batch.vertex_counts.sum()) + 10,
                   len(batch) + 3) as eng:
        for _ in range(2):
            assert np.array_equal(eng.count(batch.src, batch.dst, batch.edge_offsets,
                                            batch.vertex_counts), expected)
        got = eng.count(dev(batch.src), dev(batch.dst), batch.edge_offsets, batch.vertex_counts)
        assert np.array_equal(got, expected)
        # smaller batches through the same captured graph: a prefix, a suffix
        k = 17
        eo = batch.edge_offsets[:k + 1]
        got = eng.count(batch.src[:eo[-1]], batch.dst[:eo[-1]], eo, batch.vertex_counts[:k])
        assert np.array_equal(got, expected[:k])
        a = int(batch.edge_offsets[k])
        eo2 = batch.edge_offsets[k:] - a
        got = eng.count(batch.src[a:], batch.dst[a:], eo2, batch.vertex_counts[k:])
        assert np.array_equal(got, expected[k:])
        # one graph, then an empty batch
        s, d, n = batch.graph(3)
        assert eng.count(s, d, [0, len(s)], [n])[0] == expected[3]
        assert len(eng.count(np.zeros(0, np.int32), np.zeros(0, np.int32), [0], [])) == 0


@pytest.mark.parametrize("tuning", [
    {"warp_max_list": 0, "warp_max_partners": 0},
    {"warp_max_list": 128, "warp_max_partners": 1 << 30},
    {"warp_max_list": 16, "warp_max_partners": 8, "heavy_ratio_pct": 250},
    {"heavy_ratio_pct": 1 << 20},
])
def test_tuning_never_changes_counts(tc, batch, expected, tuning):
    import graphgen as gg

    s20, d20 = gg.rmat(14, 16 << 14, 5)
    want = oracle.forward(s20, d20, 1 << 14, per_vertex=True)
    try:
        tc.tc_set_tuning(tuning)
        assert tc.tc_get_tuning()["warp_max_list"] == tuning.get("warp_max_list", 128)
        got = tc.tc_count_batch(dev(batch.src), dev(batch.dst), batch.edge_offsets,
                                batch.vertex_counts)
        assert np.array_equal(got, expected)
        T, t, deg = tc.tc_count_per_vertex(dev(s20), dev(d20), 1 << 14)
        assert T == want["T"] and np.array_equal(t.cpu().numpy(), want["t"])
        with tc.Engine(int(batch.edge_offsets[-1]), int(batch.vertex_counts.sum()),
                       len(batch), tuning=tuning) as eng:
            assert np.array_equal(eng.count(batch.src, batch.dst, batch.edge_offsets,
                                            batch.vertex_counts), expected)
    finally:
        tc.tc_set_tuning(None)
    assert tc.tc_get_tuning() == tc.DEFAULT_TUNING


def test_batch_errors(tc, batch, expected):
    s = batch.src.copy()
    g = 7
    s[batch.edge_offsets[g]] = batch.vertex_counts[g]  # one id past its graph
    with pytest.raises(tc.TCError) as e:
        tc.tc_count_batch(dev(s), dev(batch.dst), batch.edge_offsets, batch.vertex_counts)
    assert e.value.code == tc.TC_ERR_ID_RANGE
    # only graph g fails; every other total is still exact
    want = expected.copy()
    want[g] = np.uint64(tc.TC_COUNT_ERROR)
    assert np.array_equal(e.value.totals, want)
    s[batch.edge_offsets[30] + 1] = -1  # a second bad graph, negative id
    want[30] = np.uint64(tc.TC_COUNT_ERROR)
    with tc.Engine(int(batch.edge_offsets[-1]), int(batch.vertex_counts.sum()),
                   len(batch)) as eng:
        for _ in range(2):
            with pytest.raises(tc.TCError) as e:
                eng.count(s, batch.dst, batch.edge_offsets, batch.vertex_counts)
            assert e.value.code == tc.TC_ERR_ID_RANGE
            assert np.array_equal(e.value.totals, want)
        # the error flags are cleared for the next batch
        assert np.array_equal(eng.count(batch.src, batch.dst, batch.edge_offsets,
                                        batch.vertex_counts), expected)
    bad = batch.edge_offsets.copy()
    bad[0] = 1
    with pytest.raises(tc.TCError) as e:
        tc.tc_count_batch(dev(batch.src), dev(batch.dst), bad, batch.vertex_counts)
    assert e.value.code == tc.TC_ERR_INVALID_ARG  # offsets must start at 0
    with tc.Engine(1000, 1000, 4) as eng:
        with pytest.raises(tc.TCError) as e:
            eng.count(batch.src, batch.dst, batch.edge_offsets, batch.vertex_counts)
        assert e.value.code == tc.TC_ERR_OVERFLOW
        eng.submit(np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), [0, 3], [3])
        with pytest.raises(tc.TCError):
            eng.submit(np.array([0], np.int32), np.array([1], np.int32), [0, 1], [2])
        assert eng.wait()[0] == 1
        # the engine stays usable after an id error in a batch
        with pytest.raises(tc.TCError) as e:
            eng.count(np.array([0, 5], np.int32), np.array([1, 2], np.int32), [0, 2], [3])
        assert e.value.code == tc.TC_ERR_ID_RANGE
        assert eng.count(np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32),
                         [0, 3], [3])[0] == 1
    assert len(tc.tc_count_batch(dev(batch.src[:0]), dev(batch.dst[:0]), [0], [])) == 0


def test_repeated_edges_in_batch(tc):
    """Graphs with repeats, reversed copies and self-loops, counted as one
    union: every graph's repeats meet in its own forward lists (ids of
    different graphs never share a list) and are dropped there, so each
    total equals the oracle's on that graph alone."""
    from graphgen import families as fam

    parts = [fam.random_multigraph(n, m, seed) for n, m, seed in
             [(40, 900, 1), (300, 6000, 2), (2000, 30000, 3), (7, 200, 4), (1500, 5000, 5)]]
    # a clique given in both directions, shuffled: its lists hold every entry twice
    a, b = (x.astype(np.int32) for x in np.triu_indices(120, 1))
    order = np.random.default_rng(6).permutation(2 * len(a))
    parts.append((np.concatenate([a, b])[order], np.concatenate([b, a])[order], 120))
    src = np.concatenate([p[0] for p in parts])
    dst = np.concatenate([p[1] for p in parts])
    eo = np.concatenate([[0], np.cumsum([len(p[0]) for p in parts])])
    vn = [p[2] for p in parts]
    want = np.array([oracle.forward(*p, per_vertex=False)["T"] for p in parts], np.uint64)
    assert want[-1] == 120 * 119 * 118 // 6
    assert np.array_equal(tc.tc_count_batch(dev(src), dev(dst), eo, vn), want)
    with tc.Engine(len(src) + 100, sum(vn) + 10, len(parts) + 2) as eng:
        for _ in range(2):
            assert np.array_equal(eng.count(src, dst, eo, vn), want)


def test_empty_and_tiny_graphs_in_batch(tc):
    # graphs with no edges, one edge, a triangle, K5, and isolated vertices
    parts = [([], [], 4), ([0], [1], 2), ([0, 1, 2], [1, 2, 0], 3),
             (*[list(x) for x in np.triu_indices(5, 1)], 5), ([], [], 1)]
    src = np.concatenate([np.asarray(p[0], np.int32) for p in parts])
    dst = np.concatenate([np.asarray(p[1], np.int32) for p in parts])
    eo = np.concatenate([[0], np.cumsum([len(p[0]) for p in parts])])
    vn = [p[2] for p in parts]
    want = [0, 0, 1, 10, 0]
    assert tc.tc_count_batch(dev(src), dev(dst), eo, vn).tolist() == want
    with tc.Engine(100, 100, 8) as eng:
        assert eng.count(src, dst, eo, vn).tolist() == want


def test_batch_counter_and_plain_loop(tc, batch, expected):
    from paper_1503_00576_gb300 import batching

    cap = batching.Capacity(pairs=int(batch.edge_offsets[-1]) // 5,
                            vertices=int(batch.vertex_counts.sum()) // 4, graphs=9)
    with batching.BatchCounter(cap) as bc:
        assert np.array_equal(bc.count(batch.src, batch.dst, batch.edge_offsets,
                                       batch.vertex_counts), expected)
        assert np.array_equal(bc.count(dev(batch.src), dev(batch.dst), batch.edge_offsets,
                                       batch.vertex_counts), expected)
    assert np.array_equal(batching.count_plain(dev(batch.src), dev(batch.dst),
                                               batch.edge_offsets, batch.vertex_counts),
                          expected)
    assert np.array_equal(batching.count_plain(batch.src, batch.dst, batch.edge_offsets,
                                               batch.vertex_counts), expected)


def test_autotune_picks_a_candidate(tc, batch, tmp_path, monkeypatch):
    from paper_1503_00576_gb300 import autotune, batching

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    cap = batching.Capacity(pairs=int(batch.edge_offsets[-1]),
                            vertices=int(batch.vertex_counts.sum()), graphs=len(batch))
    rec = autotune.tune_batches(dev(batch.src), dev(batch.dst), batch.edge_offsets,
                                batch.vertex_counts, cap, candidates=autotune.CANDIDATES[:3],
                                repeats=1)
    assert rec["tuning"] in autotune.CANDIDATES[:3] and not rec["cached"]
    again = autotune.tune_batches(dev(batch.src), dev(batch.dst), batch.edge_offsets,
                                  batch.vertex_counts, cap)
    assert again["cached"] and again["tuning"] == rec["tuning"]
    s, d, n = batch.graph(1)
    try:
        rec = autotune.tune_graph(dev(s), dev(d), n, candidates=autotune.CANDIDATES[:2],
                                  repeats=1)
        assert tc.tc_get_tuning() == rec["tuning"]
    finally:
        tc.tc_set_tuning(None)
