"""Host-side helpers of bench.py (no GPU): the algorithmic byte counts of the streaming
kernels, the per-shape DRAM traffic lookup and its source-hash guard, the workload
options."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402


def test_stream_bytes_counts_each_array_once():
    wl = W.dam_break_2d(dx=0.05)
    n, nf, d = wl.n_total, wl.n_fluid, 2
    ncells = 1000
    b = bench.stream_bytes(wl, ncells)
    # keys: fluid read x, u, a, xsph (8 B each per axis) + tag, write x + key; walls x + tag, key
    assert b["keys"] == nf * (4 * d * 8 + 4 + d * 8 + 4) + (n - nf) * (d * 8 + 8)
    # 10 bits of cell id: two 8-bit passes of an 8-byte (key, index) read and write
    assert b["passes"] == 2 and b["sort"] == 2 * n * 16
    # reorder: perm, key, tag, x, u, rho, m read, a read for fluid; x, u, rho, m, tag and the
    # FP32 shadow (2 x 16 B) written; a 4-byte offset read and written per cell
    assert b["reorder"] == (n * (12 + 2 * d * 8 + 16) + nf * d * 8
                            + n * (2 * d * 8 + 20 + 32) + ncells * 8)
    b64 = bench.stream_bytes(wl.with_precision(0), ncells)
    assert b64["reorder"] - b["reorder"] == n * 32  # 2 x 32 B FP64 shadow
    assert bench.stream_bytes(wl, 256)["passes"] == 1
    assert bench.stream_bytes(wl, 257)["passes"] == 2


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    t = {"source_hash": bench.source_hash(),
         "dam_break_2d": {"k_density": {"4": 123}, "k_momentum": {"4": 456, "8": 789}}}
    (prof / "traffic.json").write_text(json.dumps(t))
    h = bench.source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: h)
    assert bench.measured_traffic("dam_break_2d", "k_density", 4) == 123
    assert bench.measured_traffic("dam_break_2d", "k_momentum", 8) == 789
    assert bench.measured_traffic("dam_break_2d", "k_density", 8) is None  # shape not captured
    assert bench.measured_traffic("taylor_green_3d", "k_density", 1) is None
    t["source_hash"] = "0" * 16  # kernels changed since the capture
    (prof / "traffic.json").write_text(json.dumps(t))
    assert bench.measured_traffic("dam_break_2d", "k_density", 4) is None


def test_workload_wall_option():
    wl = bench.workload("dam_break_2d", "adami")
    assert wl.wall_bc == 1 and wl.name.endswith("_adami")
    assert "Adami" in bench.describe(wl)["workload"]
    assert bench.workload("dam_break_2d").wall_bc == 0
    batch = bench.workload("batch_tg2d", "adami")
    assert all(w.wall_bc == 1 for w in batch)


def test_workload_integrator_option():
    wl = bench.workload("dam_break_2d", "density", "pec")
    assert wl.integrator == 1 and wl.name.endswith("_pec")
    d = bench.describe(wl)
    assert "predict-evaluate-correct" in d["workload"] and "pairs_counted" in d
    assert bench.workload("dam_break_2d").integrator == 0
    assert "pairs_counted" not in bench.describe(bench.workload("dam_break_2d"))
    batch = bench.workload("batch_tg2d", "density", "pec")
    assert all(w.integrator == 1 for w in batch)
    assert "predict-evaluate-correct" in bench.describe(bench.BatchView(batch))["workload"]


def test_falling_cube_workload():
    wl = bench.workload("falling_cube_3d")
    assert wl.kernel == W.CUBIC_SPLINE and wl.n_total == 1_000_000 and wl.n_fluid == wl.n_total
    d = bench.describe(wl)
    assert "cubic spline" in d["workload"] and "paper_context" in d
    assert bench.kernel_flops(wl) == (6, 8)
