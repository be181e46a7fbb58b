"""Host logic of bench.py, on the CPU: the roofline arithmetic of the
counting phase, the committed traffic figure keyed by the kernel sources,
the clock sampler's parsing, and the reference arm's JSON line (the CPU
oracle on a bounded sample)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _prof(count_ms, other_ms, steps):
    names = ("canon", "rank", "orient", "sort", "offsets", "lists", "groups")
    prof = {k: (other_ms * steps, 3 * steps) for k in names}
    prof["count"] = (count_ms * steps, 4 * steps)
    return prof


def test_counting_roofline_bytes_rule():
    work = {"lookups": 10 ** 9, "inserts": 2 * 10 ** 8, "merge_work": 5 * 10 ** 9}
    m_in, m, n, steps = 4 * 10 ** 6, 3 * 10 ** 6, 1 << 20, 2
    r = bench.roofline(_prof(2.0, 1.0, steps), steps, m_in, m, n, "none", work)
    assert r["kernel"] == "k_count+k_count_big" and r["bound"] == "hbm"
    want = 4 * (10 ** 9 + 2 * 10 ** 8) + 4 * m + 8 * (n + 1) + 28 * n
    assert r["algorithmic_bytes_per_launch"] == want
    assert r["ms_per_launch"] == pytest.approx(2.0)
    assert r["achieved"] == pytest.approx(want / 2e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["launches_timed"] == steps
    # total-only: no per-vertex array
    t = bench.roofline(_prof(2.0, 1.0, steps), steps, m_in, m, n, "none", work, total_only=True)
    assert t["algorithmic_bytes_per_launch"] == want - 28 * n


def test_roofline_picks_the_dominant_kernel():
    work = {"lookups": 1, "inserts": 1, "merge_work": 1}
    r = bench.roofline(_prof(0.1, 5.0, 1), 1, 4096, 4096, 1 << 12, "none", work)
    assert r["kernel"] != "k_count+k_count_big"


def test_committed_traffic_needs_the_current_sources(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["rmat24"]["k_count+k_count_big"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_hash"])
    assert bench.committed_traffic("k_count+k_count_big", "rmat24") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.committed_traffic("k_count+k_count_big", "rmat24") is None
    assert bench.committed_traffic("k_count+k_count_big", "er16k") is None


def test_clock_sampler_parses_samples(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("GPU-1, 2070, 2070, 900.5, Not Active, Not Active, Not Active, Active\n"
                    "GPU-1, 2060, 2070, 901.0, Not Active, Not Active, Not Active, Not Active\n"
                    "GPU-2, 1000, 2070, 100.0, Active, Not Active, Not Active, Not Active\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.ClockSampler("GPU-1")
    c.proc, c.path = Done(), str(path)
    got = c.stop()
    assert got["sm_mhz"] == pytest.approx(2065.0) and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"] and got["samples"] == 2


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "er16k", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["steps"] == 2
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["sample_pairs_per_step"] == d["config"]["m_in"] == 131072


def test_gather_over_ranks_alone():
    import bench

    assert bench.gather_over_ranks(None, [True, False, 7]) == [[True, False, 7]]
    parts = bench.gather_over_ranks(None, [True, bool(None), 12])
    assert all(p[0] for p in parts) and not all(p[1] for p in parts)
    assert sum(p[2] for p in parts) == 12


def test_step_stats():
    import bench

    st = bench.step_stats([40.0, 42.0, 44.0, 42.0])
    assert st["mean"] == 42.0 and st["median"] == 42.0
    assert st["min"] == 40.0 and st["max"] == 44.0 and st["steps"] == 4
    assert abs(st["std"] - 2 ** 0.5) < 1e-4
    assert bench.step_stats([5.0])["std"] == 0.0


def test_run_batched_plumbing(monkeypatch):
    """run_batched's host logic with the device work faked (counts = pairs
    per graph): one rank, and two ranks of which this process is rank 0,
    through a stand-in process group whose collectives see both ranks as
    this one."""
    import types

    import numpy as np
    import torch

    import bench
    from paper_1503_00576_gb300 import autotune, batching

    def fake_count(s, d, eo, vn):
        return np.diff(np.asarray(eo, np.int64)).astype(np.uint64)

    class FakeCounter:
        def __init__(self, cap, tuning=None):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def count(self, s, d, eo, vn):
            return fake_count(s, d, eo, vn)

    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(batching, "count_plain", fake_count)
    monkeypatch.setattr(batching, "BatchCounter", FakeCounter)
    monkeypatch.setattr(autotune, "tune_batches",
                        lambda *a, **k: {"tuning": {"t": 1}, "cached": False, "ms": {}})
    args = types.SimpleNamespace(batch_graphs=24, serve_graphs=0)
    r = bench.run_batched(args, None)
    import graphgen

    m = graphgen.batch_params(24, 1005)[1]
    assert r["graphs"] == 24 and r["pairs"] == int(m.sum()) and r["triangles"] == int(m.sum())
    assert r["counts_identical"] is True and r["oracle_identical"] is None
    assert r["ranks"] == 1 and r["graphs_per_rank"] == 24 and r["served"] is None

    def all_gather(parts, t):
        for p in parts:
            p.copy_(t)

    pg = types.SimpleNamespace(get_world_size=lambda: 2, all_gather=all_gather,
                               all_reduce=lambda t, op=None: None, barrier=lambda **k: None,
                               ReduceOp=types.SimpleNamespace(MAX="max"))
    r2 = bench.run_batched(args, None, rank=0, world=2, pg=pg, dev=None)
    mine = batching.deal_graphs(np.concatenate([[0], np.cumsum(m)]), 2)[0]
    assert r2["ranks"] == 2 and r2["graphs"] == 24 and r2["pairs"] == int(m.sum())
    assert r2["triangles"] == 2 * int(m[mine].sum())  # both stand-in ranks are this one
    assert r2["counts_identical"] is True


class _FakeEvent:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 2.0


def _fake_cuda(monkeypatch):
    import types

    import torch

    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    return types


def test_run_paper_table_plumbing(monkeypatch):
    import bench

    types = _fake_cuda(monkeypatch)
    tc = types.SimpleNamespace(tc_count_host=lambda s, d, n: 11,
                               tc_count=lambda s, d, n, stream=None: 11)
    rows = [r for r in bench.PAPER_TABLE1 if r[0] in ("Kronecker 16", "Watts-Strogatz")]
    out = bench.run_paper_table(tc, rows, repeats=3)
    assert [r["graph"] for r in out] == ["Kronecker 16", "Watts-Strogatz"]
    k16, ws = out
    assert k16["n"] == 1 << 16 and k16["pairs"] == 2_500_000 and k16["triangles"] == 11
    assert k16["ms_device_resident"] == round(2.0 / 3, 3)
    assert k16["paper"] == {"edge_entries": 5e6, "triangles": 119e6, "cpu_ms": 2810,
                            "gtx980_ms": 82}
    assert ws["n"] == 1_000_000 and ws["pairs"] == 25_000_000
    assert "seed 1116" in k16["input"] and "Watts-Strogatz" in ws["input"]


def test_run_paper_format_plumbing(monkeypatch):
    import numpy as np
    import torch

    import bench

    types = _fake_cuda(monkeypatch)
    n = 5
    t_ref = torch.arange(n, dtype=torch.int64)
    deg_ref = torch.arange(n, dtype=torch.int32) + 1
    seen = []

    def per_vertex(s, d, nn, stream=None, t_out=None, deg_out=None):
        seen.append(int(s.numel()))
        t_out.copy_(t_ref)
        deg_out.copy_(deg_ref)
        return 7, t_out, deg_out

    tc = types.SimpleNamespace(tc_count_per_vertex=per_vertex)
    s = torch.tensor([0, 1, 2], dtype=torch.int32)
    d = torch.tensor([1, 2, 0], dtype=torch.int32)
    r = bench.run_paper_format(4, tc, s, d, n, 3, 7, t_ref, deg_ref, None)
    assert set(seen) == {6} and len(seen) == 3 + 4
    assert r["pairs"] == 6 and r["edges"] == 3 and r["identical_to_main_run"] is True
    assert abs(r["ms_per_step"] - 0.5) < 1e-9 and r["pairs_per_s"] == 6 / 0.0005
    with np.testing.assert_raises(AssertionError):
        bench.run_paper_format(1, tc, s, d, n, 3, 8, t_ref, deg_ref, None)  # T differs
