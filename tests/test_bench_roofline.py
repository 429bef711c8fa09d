"""Host arithmetic of bench.py's measurement: the derived FP32 peak, the pair-sort pass count and
the kernels one step launches, the per-stage roofline table and the composite T*/T, and the rule
that measured DRAM traffic is reported only for the build and workload it was captured on."""
import math
import types

import pytest

import bench


def test_fp32_peak_from_sm_count_and_clock():
    # 152 SMs x 128 FP32 lanes x 2 (FMA) at 2.07 GHz: the 80.5 TFLOP/s of a GB300
    cp = bench.compute_peaks({"sm_max_mhz": 2070.0}, 152)
    assert cp["fp32_tflops"] == pytest.approx(80.548, abs=1e-3)
    # 4 MUFU results per sub-partition and clock
    assert cp["sfu_tops"] == pytest.approx(152 * 16 * 2.07 / 1e3)


@pytest.mark.parametrize("tiles,passes", [(1, 0), (2, 1), (256, 1), (257, 1), (512, 1), (513, 2),
                                          (23920, 2), (65536, 2), (131073, 2), (262145, 3)])
def test_tile_sort_passes(tiles, passes):
    """8-bit digits, or 9-bit ones where they save a pass: ceil(b/8) vs ceil(b/9) for b id bits."""
    assert bench.tile_sort_passes(types.SimpleNamespace(total_tiles=tiles)) == passes


def test_kernels_per_step_of_the_bench_workload():
    # 16 x 16 tiles over 2 x {640x480, 960x540, 1280x720, 1280x1024}
    tiles = sum(math.ceil(w / 16) * math.ceil(h / 16) for w, h in bench.SIZES)
    assert tiles == 23920
    # the ncu launch list of one graph-replayed step counts 38 launches
    assert bench.kernels_per_step(types.SimpleNamespace(total_tiles=tiles)) == 38


def _workload():
    return {"n": 1000, "views": 8, "pairs": 20_000, "visible_entries": 3000, "visible_gaussians": 700,
            "depth_sort_passes": 4, "tile_sort_passes": 2, "frag_fwd_eval": 1_000_000, "frag_fwd_add": 400_000,
            "frag_bwd_eval": 1_200_000, "frag_bwd_add": 400_000}


def test_roofline_table_fractions_and_lower_bounds():
    pk = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}
    stage = {"project": 0.01, "bin_sort": 0.05, "render_fwd": 0.02, "composite_bwd": 0.04,
             "project_bwd_adam": 0.03}
    t = bench.roofline_table(stage, _workload(), pk, 100)
    fp32 = 100 * 128 * 2 * 2.0 / 1e3   # TFLOP/s
    for k in ("project", "bin_sort", "project_bwd_adam"):
        r = t[k]
        assert r["bound"] == "hbm" and r["unit"] == "GB/s"
        # achieved = bytes / time; frac = achieved / peak; the lower bound is bytes at the peak
        assert r["achieved"] == pytest.approx(r["bytes"] / (stage[k] * 1e-3) / 1e9, abs=0.06)
        assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, abs=1e-4)
        assert r["t_star_ms"] == pytest.approx(r["bytes"] / 6000.0 / 1e6, abs=1e-4)
    # every visible row moves its parameters and both Adam moments in and out (6 x 236 B)
    assert t["project_bwd_adam"]["bytes"] >= 6 * 236 * 700
    for k, per in (("render_fwd", 20), ("composite_bwd", 60)):
        r = t[k]
        w = _workload()
        ev = w["frag_fwd_eval"] if k == "render_fwd" else w["frag_bwd_eval"]
        assert r["bound"] == "alu" and r["flops"] == per * ev
        assert r["peak"] == pytest.approx(fp32, abs=0.05)
        assert r["frac"] == pytest.approx(r["flops"] / (stage[k] * 1e-3) / 1e12 / fp32, abs=1e-4)
        # the lower bound is the larger of the FP32 and the SFU (one exponential per fragment) times
        sfu = 100 * 16 * 2.0 / 1e3
        assert r["t_star_ms"] == pytest.approx(max(r["flops"] / fp32 / 1e9, r["sfu_ops"] / sfu / 1e9), abs=1e-4)


def test_composite_fraction_is_sum_of_lower_bounds_over_step():
    table = {"a": {"t_star_ms": 0.1}, "b": {"t_star_ms": 0.25}, "c": {"t_star_ms": 0.15}}
    c = bench.composite_fraction(table, 2.0)
    assert c["t_star_ms"] == pytest.approx(0.5)
    assert c["frac"] == pytest.approx(0.25)


def test_traffic_only_for_the_captured_build_and_workload(monkeypatch):
    cur = bench.source_digest()
    monkeypatch.setattr(bench, "TRAFFIC", {"digest": cur, "n": 2_000_000, "tile": 16, "chunk": 256,
                                           "bytes": {"composite_bwd": 123}})
    assert bench.stage_traffic("composite_bwd", 16, 256, 2_000_000) == 123
    assert bench.stage_traffic("render_fwd", 16, 256, 2_000_000) is None
    assert bench.stage_traffic("composite_bwd", 8, 256, 2_000_000) is None
    assert bench.stage_traffic("composite_bwd", 16, 128, 2_000_000) is None
    assert bench.stage_traffic("composite_bwd", 16, 256, 1_000_000) is None
    monkeypatch.setattr(bench, "TRAFFIC", {"digest": "0" * 64, "n": 2_000_000, "tile": 16, "chunk": 256,
                                           "bytes": {"composite_bwd": 123}})
    assert bench.stage_traffic("composite_bwd", 16, 256, 2_000_000) is None


def test_source_digest_covers_every_cuda_source_and_the_header():
    import glob
    import hashlib
    import os
    root = os.path.dirname(os.path.abspath(bench.__file__))
    files = sorted(glob.glob(os.path.join(root, "paper_2604_12942_gb300", "csrc", "*.cu*")))
    assert any(f.endswith("render.cu") for f in files) and any(f.endswith(".cuh") for f in files)
    h = hashlib.sha256()
    for f in files + [os.path.join(root, "include", "gs.h")]:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    assert bench.source_digest() == h.hexdigest()
