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
