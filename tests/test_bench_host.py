"""bench.py's host-side helpers (CPU only): the algorithmic-byte formulas of
the roofline, the traffic record that is only trusted while the kernel's
sources are unchanged, and the workload overrides."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_formulas():
    st = {"cand_ids": 1000, "gathered_rows": 300, "proposals": 50, "merges": 7, "K": 20}
    # ids 4 B; rows dp*4 B + an 8 B worst-key snapshot; proposals 8 B
    assert bench.join_bytes(st, 16) == 1000 * 4 + 300 * (16 * 4 + 8) + 50 * 8
    # proposals read 8 B; each merged list read and written
    assert bench.merge_bytes(st) == 50 * 8 + 7 * 2 * 20 * 8


def test_traffic_record_needs_matching_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    rec = {"k": {"dram_bytes_per_launch": 123, "sources": ["k.cu"],
                 "sources_sha256": hashlib.sha256(b"kernel v1").hexdigest()}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k") == 123
    src.write_text("kernel v2")  # the kernel changed since the capture
    assert bench.measured_traffic("k") is None
    assert bench.measured_traffic("missing") is None


def test_workload_overrides_are_named():
    class A:
        workload, n, rho, delta, max_iters = "uniform_n2k_d8", 500, 0.5, None, 4
    w, x, name = bench._workload(A())
    assert (w.n, w.rho, w.max_iters) == (500, 0.5, 4) and x.shape == (500, 8)
    assert name == "uniform_n2k_d8_n500_rho0.5_max_iters4"


@pytest.mark.parametrize("ranks", [1, 2, 3, 8])
def test_batched_data_sets_dealt_by_cost(ranks):
    """Every data set of the batched workload lands on exactly one rank, and
    the heaviest rank's n*d load is within one data set of the mean."""
    import workloads
    specs = workloads.batched_specs(256, 0)
    costs = [s["n"] * s["d"] for s in specs]
    parts = bench.deal_by_cost(costs, ranks)
    assert len(parts) == ranks
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= sum(costs) / ranks + max(costs)
    if ranks > 1:
        # the deal is balanced far better than round-robin's worst case
        assert max(loads) - min(loads) <= max(costs)


def test_deal_by_cost_hand_case():
    """Largest first to the least-loaded rank: costs 7, 5, 4, 3, 1 over two
    ranks give {7, 3} and {5, 4, 1}, loads 10 and 10."""
    assert bench.deal_by_cost([4, 7, 1, 5, 3], 2) == [[1, 4], [0, 2, 3]]
