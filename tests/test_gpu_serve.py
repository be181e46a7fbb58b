"""Serving loop: every request of a mixed, randomly timed stream gets
exactly the count of its graph alone.

Requests arrive at seeded Poisson times, from host memory and from graphs
registered on the device, interleaved with requests the server must refuse
(too large for an engine, ids out of range).  The refused ones fail alone;
every other result equals the oracle's count (small graphs) and tc_count's
on the same graph.  Integer counts: the tolerance is zero.
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
def mix():
    return graphgen.graph_batch(40, 21, log2_n=(4, 12), degree=(1.0, 48.0))


@pytest.fixture(scope="module")
def expected(mix):
    return [oracle.forward(*mix.graph(g), per_vertex=False)["T"] for g in range(len(mix))]


def test_poisson_mix_equals_alone(tc, mix, expected):
    import torch

    from paper_1503_00576_gb300 import batching, serve

    cap = batching.Capacity(pairs=int(np.diff(mix.edge_offsets).max()) * 3,
                            vertices=int(mix.vertex_counts.max()) * 3, graphs=8)
    rng = np.random.default_rng(5)
    big_s = np.arange(cap.pairs + 1, dtype=np.int32) % 50
    big_d = (big_s + 1) % 50
    with serve.Server(cap, engines=2) as srv:
        handles = {g: srv.register(*mix.graph(g)) for g in range(0, len(mix), 4)}
        futs, want = [], []
        for g in rng.permutation(len(mix)):
            s, d, n = mix.graph(int(g))
            if g in handles and rng.random() < 0.7:
                futs.append(srv.submit_resident(handles[g]))
            elif rng.random() < 0.5:
                futs.append(srv.submit(torch.from_numpy(s.copy()).pin_memory(),
                                       torch.from_numpy(d.copy()).pin_memory(), n))
            else:
                futs.append(srv.submit(s, d, n))
            want.append(expected[g])
            if rng.random() < 0.1:
                futs.append(srv.submit(big_s, big_d, 50))  # more pairs than an engine holds
                want.append("overflow")
            if rng.random() < 0.1:
                futs.append(srv.submit(s[:3], np.full(3, n, np.int32), n))  # id n is out of range
                want.append("id_range")
            pause = rng.exponential(2e-4)
            if pause > 1e-4:
                import time

                time.sleep(pause)
        srv.drain(timeout=120)
        for f, w in zip(futs, want):
            if w == "overflow":
                with pytest.raises(tc.TCError) as e:
                    f.result()
                assert e.value.code == tc.TC_ERR_OVERFLOW
            elif w == "id_range":
                with pytest.raises(tc.TCError) as e:
                    f.result()
                assert e.value.code == tc.TC_ERR_ID_RANGE
            else:
                assert f.result() == w
        st = srv.stats()
        assert st["requests"] == sum(1 for w in want if w != "overflow")
        assert "id_range" in want and "overflow" in want
        assert st["batches"] >= 1 and st["p99_ms"] >= st["p50_ms"] > 0
    # and alone through the single-graph entry point
    for g in range(0, len(mix), 3):
        s, d, n = mix.graph(g)
        assert tc.tc_count(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n) == \
            expected[g]


def test_serve_larger_graphs_and_store_budget(tc):
    import torch

    from paper_1503_00576_gb300 import batching, serve

    graphs = [(*graphgen.rmat_graph(n, m, seed), n) for n, m, seed in
              [(1 << 14, 1 << 17, 3), (1 << 12, 40000, 4), (1 << 15, 1 << 18, 5)]]
    cap = batching.Capacity(pairs=1 << 19, vertices=1 << 16, graphs=4)
    with serve.Server(cap, engines=2, store_bytes=8 * (1 << 17) + 8 * 40000) as srv:
        h0 = srv.register(*graphs[0])
        h1 = srv.register(*graphs[1])
        with pytest.raises(tc.TCError) as e:
            srv.register(*graphs[2])  # over the resident budget
        assert e.value.code == tc.TC_ERR_OOM
        srv.unregister(h1)
        h2 = srv.register(*graphs[1])
        futs = [srv.submit(*g) for g in graphs] + [srv.submit_resident(h) for h in (h0, h2)]
        want = [tc.tc_count(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
                for s, d, n in graphs]
        assert [f.result(timeout=120) for f in futs] == want + [want[0], want[1]]
        assert want[0] == oracle.forward(*graphs[0], per_vertex=False)["T"]
