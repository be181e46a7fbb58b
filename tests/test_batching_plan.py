"""Sub-batch planning (host logic, no GPU)."""
import numpy as np
import pytest

from paper_1503_00576_gb300.batching import Capacity, plan_subbatches


def check(eo, vn, cap, plan):
    covered = []
    for first, last, fits in plan:
        covered.extend(range(first, last))
        pairs = eo[last] - eo[first]
        verts = int(np.sum(vn[first:last]))
        if fits:
            assert pairs <= cap.pairs and verts <= cap.vertices and last - first <= cap.graphs
        else:
            assert last - first == 1
            assert pairs > cap.pairs or verts > cap.vertices
    assert covered == list(range(len(vn)))


@pytest.mark.parametrize("seed", range(6))
def test_plan_covers_in_order_within_capacity(seed):
    rng = np.random.default_rng(seed)
    G = int(rng.integers(1, 400))
    m = rng.integers(0, 5000, G)
    m[rng.random(G) < 0.03] = 50_000  # some graphs larger than an engine
    vn = rng.integers(1, 3000, G).astype(np.int32)
    eo = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    cap = Capacity(pairs=20_000, vertices=40_000, graphs=int(rng.integers(1, 50)))
    plan = plan_subbatches(eo, vn, cap)
    check(eo, vn, cap, plan)
    # greedy: a fitting sub-batch could not take its successor too
    for (f, l, fits), nxt in zip(plan, plan[1:]):
        if fits and nxt[2]:
            grow = l + 1
            assert (eo[grow] - eo[f] > cap.pairs or np.sum(vn[f:grow]) > cap.vertices
                    or grow - f > cap.graphs)


def test_plan_edge_cases():
    cap = Capacity(pairs=10, vertices=10, graphs=3)
    assert plan_subbatches(np.array([0]), np.array([], np.int32), cap) == []
    eo = np.array([0, 0, 0, 0, 0])
    plan = plan_subbatches(eo, np.array([1, 1, 1, 1], np.int32), cap)
    assert plan == [(0, 3, True), (3, 4, True)]


# ------------------------------------------------------------ graphs dealt to devices
@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_deal_graphs_covers_and_balances(parts):
    import graphgen
    from paper_1503_00576_gb300.batching import deal_graphs

    vn, m, _, _ = graphgen.batch_params(4096, 1005)
    eo = np.concatenate([[0], np.cumsum(m)])
    shares = deal_graphs(eo, parts)
    assert len(shares) == parts
    assert np.array_equal(np.sort(np.concatenate(shares)), np.arange(len(vn)))
    for sh in shares:
        assert np.all(np.diff(sh) > 0)
    m = np.diff(np.asarray(eo, np.int64))
    load = np.array([m[sh].sum() for sh in shares])
    # largest-first dealing: no part exceeds the mean by more than the largest graph
    assert load.max() - load.mean() <= m.max()
    assert load.max() <= 1.02 * load.mean()


def test_deal_graphs_edge_cases():
    from paper_1503_00576_gb300.batching import deal_graphs

    assert [len(x) for x in deal_graphs(np.array([0]), 3)] == [0, 0, 0]
    # one huge graph and many small: the huge one stands alone
    eo = np.concatenate([[0], np.cumsum([1000] + [10] * 20)])
    a, b = deal_graphs(eo, 2)
    assert list(a) == [0] and list(b) == list(range(1, 21))
    with pytest.raises(ValueError):
        deal_graphs(eo, 0)


def test_gather_graphs_numpy_and_torch():
    import torch

    from paper_1503_00576_gb300.batching import gather_graphs

    eo = np.array([0, 3, 3, 7, 9], np.int64)
    vn = np.array([4, 1, 5, 2], np.int32)
    src = np.arange(9, dtype=np.int32)
    dst = src + 100
    s, d, e, v = gather_graphs(src, dst, eo, vn, [0, 2, 3])
    assert list(s) == [0, 1, 2, 3, 4, 5, 6, 7, 8] and list(d) == list(range(100, 109))
    assert list(e) == [0, 3, 7, 9] and list(v) == [4, 5, 2]
    s, d, e, v = gather_graphs(torch.from_numpy(src), torch.from_numpy(dst), eo, vn, [3, 1])
    assert s.tolist() == [7, 8] and d.tolist() == [107, 108]
    assert list(e) == [0, 2, 2] and list(v) == [2, 1]
    s, d, e, v = gather_graphs(src, dst, eo, vn, [])
    assert len(s) == 0 and list(e) == [0] and len(v) == 0
