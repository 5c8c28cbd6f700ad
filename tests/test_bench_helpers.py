"""Host-side arithmetic of bench.py (no GPU): roofline helpers, whole-job
throughput, algorithmic byte counts."""
import bench


def test_issue_and_traffic_views_follow_the_captured_source(monkeypatch):
    units = {"fwd_warp_visits": 1000, "bwd_warp_visits": 2000, "fwd_composited": 10, "bwd_composited": 10}
    monkeypatch.setattr(bench, "_blend_source_matches", lambda: True)
    v = bench.blend_issue("composite_bwd", units, 1.0, 2070.0)
    assert v["warp_instr_per_launch"] == int(bench.BLEND_ISSUE["composite_bwd"] * 2000)
    assert abs(v["peak"] - 152 * 4 * 2070e6 / 1e12) < 1e-3
    assert abs(v["frac"] - v["achieved"] / v["peak"]) < 1e-3
    assert bench.blend_traffic("composite_fwd", units) == int(bench.BLEND_TRAFFIC["composite_fwd"] * 10)
    # a changed kernel source voids the captured figures
    monkeypatch.setattr(bench, "_blend_source_matches", lambda: False)
    assert bench.blend_issue("composite_bwd", units, 1.0, 2070.0) is None
    assert bench.blend_traffic("composite_fwd", units) is None


def test_source_check_reads_the_kernel_file():
    # the hash is of the committed blending source; either outcome is a bool
    assert bench._blend_source_matches() in (True, False)


def test_job_value_and_flops():
    assert bench.job_value(2, 64, 10, 500.0) == 2 * 64 * 10 / 0.5
    u = {"fwd_support": 3, "fwd_composited": 2, "fwd_candidates": 5, "bwd_support": 7, "bwd_composited": 11,
         "bwd_candidates": 0}
    f = bench.FLOPS_PER_UNIT
    assert bench.blend_flops(u, "composite_fwd") == f["support"] * 3 + f["fwd_composited"] * 2 + f["candidate"] * 5
    assert bench.blend_flops(u, "composite_bwd") == f["support"] * 7 + f["bwd_composited"] * 11


def test_stage_bytes_are_per_unit_sums():
    c = {"P": 100, "F": 40, "Nb": 10, "K": 80, "Kb": 20}
    assert bench.stage_bytes("resolve", c, 5, 6, 1) == 20 * 100
    assert bench.stage_bytes("composite_fwd", c, 5, 6, 1) == 56 * 80 + 20 * 20 + 24 * 100
    assert bench.stage_bytes("raster", c, 5, 6, 2) == 12 * 6 * 5 * 2 + 8 * 100
