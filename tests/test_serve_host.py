"""Host logic of the serving loop (serve.py), on the CPU: admission by an
engine's capacity, the batches it forms (the longest prefix of waiting
requests of one kind that fits), per-request results and errors, and the
latency statistics.  The engines themselves are GPU code
(tests/test_gpu_serve.py)."""
import collections
import threading

import pytest

import paper_1503_00576_gb300 as tc
from paper_1503_00576_gb300 import serve
from paper_1503_00576_gb300.batching import Capacity


def _server(cap):
    s = serve.Server.__new__(serve.Server)  # no engines: the loop is not started
    s.cap = cap
    s._queue = collections.deque()
    s._cv = threading.Condition()
    s._done, s._outstanding, s._t0, s._batches = [], 0, None, 0
    return s


def _req(pairs, n, on_host=True, t=0.0):
    return serve._Req(None, None, n, pairs, on_host, t)


def test_oversized_requests_are_refused():
    s = _server(Capacity(pairs=100, vertices=50, graphs=4))
    f = s._admit(_req(101, 10))
    with pytest.raises(tc.TCError) as e:
        f.result(timeout=1)
    assert e.value.code == tc.TC_ERR_OVERFLOW
    f = s._admit(_req(10, 51))
    with pytest.raises(tc.TCError):
        f.result(timeout=1)
    assert not s._queue and s._outstanding == 0
    s._admit(_req(100, 50))
    assert len(s._queue) == 1 and s._outstanding == 1


def test_batches_are_prefixes_that_fit():
    s = _server(Capacity(pairs=100, vertices=60, graphs=3))
    for pairs, n, host in [(40, 10, True), (40, 10, True), (30, 10, True),   # 3rd: pairs > 100
                           (10, 10, True), (5, 5, False), (5, 5, False)]:
        s._admit(_req(pairs, n, host))
    b, kind = s._take_batch()
    assert [r.pairs for r in b] == [40, 40] and kind is True
    b, kind = s._take_batch()
    assert [r.pairs for r in b] == [30, 10] and kind is True  # stops at the other kind
    b, kind = s._take_batch()
    assert [r.pairs for r in b] == [5, 5] and kind is False
    assert not s._queue
    for _ in range(5):
        s._admit(_req(1, 1))
    b, _ = s._take_batch()
    assert len(b) == 3  # at most cap.graphs per batch


def test_results_errors_and_stats():
    s = _server(Capacity(pairs=100, vertices=100, graphs=8))
    reqs = [_req(1, 3, t=0.0), _req(1, 3, t=0.0), _req(1, 3, t=0.0)]
    for r in reqs:
        s._admit(r)
    s._finish(reqs, [7, tc.TC_COUNT_ERROR, 0])
    assert reqs[0].future.result() == 7 and reqs[2].future.result() == 0
    with pytest.raises(tc.TCError) as e:
        reqs[1].future.result()
    assert e.value.code == tc.TC_ERR_ID_RANGE
    st = s.stats(reset=True)
    assert st["requests"] == 3 and st["p50_ms"] >= 0.0 and st["p99_ms"] >= st["p50_ms"]
    assert s.stats() == {"requests": 0}
    assert s._outstanding == 0
