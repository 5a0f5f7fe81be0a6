"""Host logic of bench.py: roofline arithmetic, DRAM traffic scaling, launch count, clock parsing."""
import json
import os
import types

import numpy as np
import pytest

import bench


def _res(stage_ms, sort_design="depth_first"):
    stages = list(stage_ms)
    return dict(N=10_000_000, instances=17_000_000, W=1920, H=1080, stages=stages, sort_design=sort_design,
                visible=1.0,
                stage_ms=np.array([stage_ms[k] for k in stages]),
                pairs={"blended": 6e7, "fwd_pairs": 4e9, "bwd_pairs": 2.5e9, "fwd_pairs_masked": 6e8,
                       "bwd_pairs_masked": 4e8})


def _hbm_peak():
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p)).get("hbm_gbs", 6800.0) if os.path.exists(p) else 6800.0


def test_rooflines_hbm_and_issue_stages():
    ms = {"preprocess": 0.4, "bin_sort": 1.3, "render_fwd": 2.0, "loss": 0.13, "blend_bwd": 1.8,
          "project_bwd_adam": 2.4}
    issue = {"fp32_tops": 39.0, "mufu_tops": 10.0, "sms": 152}
    dom, out = bench.rooflines(_res(ms), "iso10M-1080p", issue)
    assert dom is out["project_bwd_adam"]  # the largest share
    peak = _hbm_peak()
    # projection backward + Adam: read and write params, m, v (6 x 236 B) + 44 B per Gaussian
    ach = 10_000_000 * (236 * 6 + 44) / 2.4e-3 / 1e9
    assert out["project_bwd_adam"]["achieved"] == pytest.approx(ach, rel=1e-3)
    assert out["project_bwd_adam"]["frac"] == pytest.approx(ach / peak, rel=1e-3)
    # issue-bound stages: pairs inside the block masks x FP32 slots per pair against the measured rate
    fwd = 6e8 * bench.FWD_SLOTS_PER_PAIR / 2.0e-3 / 1e12
    assert out["render_fwd"]["bound"] == "alu" and out["render_fwd"]["achieved"] == pytest.approx(fwd, rel=1e-3)
    assert out["render_fwd"]["frac"] == pytest.approx(fwd / 39.0, rel=1e-3)
    assert abs(sum(v["share"] for v in out.values()) - 1.0) < 1e-3
    # preprocess: 15 parameter planes read, 60 B of records written per Gaussian
    assert out["preprocess"]["achieved"] == pytest.approx(10_000_000 * 300 / 0.4e-3 / 1e9, rel=1e-3)


def test_rooflines_with_the_projection_fused_into_adam():
    ms = {"preprocess": 0.001, "bin_sort": 1.3, "render_fwd": 2.0, "loss": 0.13, "blend_bwd": 1.8,
          "project_bwd_adam": 2.5}
    res = _res(ms)
    res["fused_pre"] = True
    dom, out = bench.rooflines(res, "iso10M-1080p", None)
    assert "preprocess" not in out and dom is out["project_bwd_adam"]
    ach = 10_000_000 * (236 * 6 + 44 + 60) / 2.5e-3 / 1e9
    assert out["project_bwd_adam"]["achieved"] == pytest.approx(ach, rel=1e-3)
    assert out["project_bwd_adam"]["traffic"] == round(bench.TRAFFIC_PER_UNIT["project_bwd_adam_next"][1] * 1e7)
    frame = types.SimpleNamespace(n_tiles=120 * 68, units=types.SimpleNamespace(n=1), use_masks=True)
    assert bench.kernel_launch_count(frame, 0.2, True) == bench.kernel_launch_count(frame, 0.2) - 1


def test_traffic_scales_by_units_and_only_for_the_captured_workload():
    ms = {"preprocess": 0.4, "bin_sort": 1.3, "render_fwd": 2.0, "loss": 0.13, "blend_bwd": 1.8,
          "project_bwd_adam": 2.4}
    _, out = bench.rooflines(_res(ms), "iso10M-1080p", None)
    for name, entry in bench.TRAFFIC_PER_UNIT.items():
        if name not in out:  # the fused variant's entry (tested below)
            continue
        if entry is None:  # kernels changed since their counters were taken: no traffic figure
            assert out[name]["traffic"] is None
            continue
        unit, per, _ = entry
        n = {"gaussian": 10_000_000, "instance": 17_000_000, "pixel": 1920 * 1080, "fwd_pair": 4e9,
             "bwd_pair": 2.5e9}[unit]
        assert out[name]["traffic"] == round(per * n)
    # the sort's figure was taken on the depth-first design only
    _, glob = bench.rooflines(_res(ms, "global"), "iso10M-1080p", None)
    assert glob["bin_sort"]["traffic"] is None and glob["preprocess"]["traffic"] is not None
    _, other = bench.rooflines(_res(ms), "iso1M-1080p", None)
    assert all(v["traffic"] is None for v in other.values())
    _, rnd = bench.rooflines(_res(ms), "iso10M-1080p", None, random_order=True)
    assert all(v["traffic"] is None for v in rnd.values())


def test_launch_count_of_one_step():
    frame = types.SimpleNamespace(n_tiles=120 * 68, units=types.SimpleNamespace(n=1), use_masks=True,
                                  sort_design="global")
    # preprocess 1; sort 3 + 1 + 3 x 5 passes + 1; schedule 7; forward 3; loss 4; backward 1; Adam 2
    assert bench.kernel_launch_count(frame, 0.2) == 38
    frame.use_masks = False
    assert bench.kernel_launch_count(frame, 0.0) == 1 + 20 + 1 + 3 + 1 + 2
    # depth-first sort: visibility scan + compaction 3, depth passes 12, instance counts + their scan +
    # emission 3, two instance passes over the 13 tile bits 6, ranges 1
    frame.sort_design, frame.use_masks = "depth_first", True
    assert bench.kernel_launch_count(frame, 0.2) == 1 + 25 + 7 + 3 + 4 + 1 + 2
    # unit | tile ids over 16 bits: the global sort's chain
    frame.units.n = 16
    assert bench.kernel_launch_count(frame, 0.2) == 1 + (3 + 1 + 3 * 6 + 1) + 7 + 3 + 4 + 1 + 2


def test_clock_parsing():
    c = bench.ClockSampler("GPU-abc")
    c.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: None, kill=lambda: None)
    c.t = types.SimpleNamespace(join=lambda timeout=None: None)
    c.lines = ["0, GPU-abc, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, GPU-abc, 2050, 2070, 1300.5, 0x4, Not Active, Not Active, Not Active, Active",
               "1, GPU-other, 100, 2070, 10.0, 0x0, Active, Not Active, Not Active, Not Active"]
    r = c.stop()
    assert r["samples"] == 2 and r["sm_max_mhz"] == 2070 and r["reasons"] == ["sw_power_cap"]
    assert r["sm_mhz"] == pytest.approx(2060.0)
