"""The multi-rank path of count_sharded on CPU: two gloo ranks, each with
its share of the counts, must both end with the whole T, t and deg.

The shares come from the CPU oracle (a stand-in for tc_count_part /
tc_count_per_vertex_part, which need a GPU): rank r holds t(v) for the
vertices v = r mod 2 and a split of T.  What is tested is the host logic
around the shares -- which share a rank asks for, and the sum all-reduce
that joins them -- over a real two-process gloo group (127.0.0.1)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, port: int, per_vertex: bool):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import graphgen
    import oracle
    from paper_1503_00576_gb300.shard import count_sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        src, dst = graphgen.er(300, 3000, 17)
        n = 300
        want = oracle.forward(src, dst, n)
        asked = []

        def share_total(s, d, nn, part, parts, stream=None):
            asked.append((part, parts))
            return want["T"] // parts + (want["T"] % parts if part == 0 else 0)

        def share_pv(s, d, nn, part, parts, stream=None):
            asked.append((part, parts))
            t = torch.from_numpy(want["t"].astype(np.int64))
            t[torch.from_numpy(np.arange(nn) % parts != part)] = 0
            return share_total(s, d, nn, part, parts), t, torch.from_numpy(want["deg"])

        s, d = torch.from_numpy(src), torch.from_numpy(dst)
        if per_vertex:
            T, t, deg = count_sharded(s, d, n, per_vertex=True, count_part=share_pv)
            assert np.array_equal(t.numpy(), want["t"])
            assert np.array_equal(deg.numpy(), want["deg"])
        else:
            T = count_sharded(s, d, n, count_part=share_total)
        assert T == want["T"], (T, want["T"])
        assert asked[0] == (rank, WORLD)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("per_vertex", [False, True])
def test_two_gloo_ranks_sum_their_shares(per_vertex):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.start_processes(_worker, args=(_free_port(), per_vertex), nprocs=WORLD, join=True,
                       start_method="spawn")


def _batch_worker(rank: int, port: int):
    """Two ranks deal a batch by size, each generates and counts only its
    graphs (the oracle stands in for the GPU engines) and the verdicts and
    triangle sums are joined as bench.py joins them."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import graphgen
    import oracle
    from paper_1503_00576_gb300.batching import deal_graphs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        G, seed, sizes = 48, 91, (5, 10)
        _, m, _, _ = graphgen.batch_params(G, seed, log2_n=sizes)
        shares = deal_graphs(np.concatenate([[0], np.cumsum(m)]), WORLD)
        mine = shares[rank]
        gb = graphgen.graph_batch(G, seed, log2_n=sizes, only=mine, threads=2)
        got = [oracle.forward(*gb.graph(j), per_vertex=False)["T"] for j in range(len(gb))]
        full = graphgen.graph_batch(G, seed, log2_n=sizes, threads=2)
        want = [oracle.forward(*full.graph(g), per_vertex=False)["T"] for g in range(G)]
        ok = got == [want[g] for g in mine]
        parts = bench.gather_over_ranks(dist, [ok, sum(got), len(mine)])
        assert [p[0] for p in parts] == [1, 1]
        assert sum(p[1] for p in parts) == sum(want)
        assert sum(p[2] for p in parts) == G
        assert parts[rank] == [1, sum(got), len(mine)]
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_count_their_graphs():
    mp = pytest.importorskip("torch.multiprocessing")
    mp.start_processes(_batch_worker, args=(_free_port(),), nprocs=WORLD, join=True,
                       start_method="spawn")
