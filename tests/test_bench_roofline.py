"""The roofline arithmetic of bench.py on hand-made level counts: the op model
(draws, holding times, still tests, jumps, walk ends), the ALU peak from the
SM count, lanes and clock, and the gather bytes against the HBM peak."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _level(walks, jumps, still, coarse=False, launches=1):
    return {"walks": walks, "jumps": jumps, "still_walks": still, "coarse": coarse,
            "launches": launches}


def test_op_model_counts_each_part_once():
    # 400 walks, 100 of them jump, 150 jumps in all, at l0 and at a coarse level.
    lv0 = _level(400, 150, 300)
    lv1 = _level(400, 150, 300, coarse=True)
    draws = 150 + 400 / 4                      # one per jump + one block per four walks
    holds = (400 + 150) - 300                  # every event but a still walk's first
    want0 = (42 * draws + 31 * holds + 2 * 400 + 15 * 150 + 24 * 100 + 1 * 300)
    want1 = (42 * draws + 31 * holds + 2 * 400 + 22 * 150 + 31 * 100 + 1 * 300)
    walk_s = 1e-3
    clocks = {"sm_mhz": 2000.0}
    peaks = {"hbm_gbs": 8000.0}
    r = bench.walk_roofline([lv0, lv1], walk_s, clocks, peaks, total_ms=2.0, num_sms=152)
    assert r["achieved"] == pytest.approx((want0 + want1) / walk_s / 1e9, rel=1e-12)
    assert r["peak"] == pytest.approx(152 * 128 * 2000.0 * 1e6 / 1e9, rel=1e-12)
    other = bench.walk_roofline([lv0, lv1], walk_s, clocks, peaks, total_ms=2.0, num_sms=148)
    assert other["peak"] == pytest.approx(148 * 128 * 2000.0 * 1e6 / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)
    assert r["ops_per_event"] == pytest.approx((want0 + want1) / (2 * 550), rel=1e-12)
    assert r["walk_kernel_share_of_step_time"] == pytest.approx(0.5)
    assert r["avg_launch_ms"] == pytest.approx(0.5)
    # gathers: 32 B per jump and 4 B per walk that jumped
    g = 2 * (32 * 150 + 4 * 100)
    assert r["gather"]["achieved"] == pytest.approx(g / walk_s / 1e9, rel=1e-12)
    assert r["gather"]["frac"] == pytest.approx(r["gather"]["achieved"] / 8000.0, rel=1e-12)
    # the capture's DRAM bytes and issue figures describe one kernel and
    # workload: reported only when the caller says the line is that one
    assert r["traffic"] is None and r["issue"] is None
    c = bench.walk_roofline([lv0, lv1], walk_s, clocks, peaks, total_ms=2.0, num_sms=152,
                            proposal=True, capture=True)
    assert c["traffic"] == bench.TRAFFIC_CAPTURE and c["issue"] == bench.ISSUE_CAPTURE
    assert r["bound"] == "alu" and r["unit"] == "Gop/s"


def test_a_walk_that_never_jumps_costs_a_quarter_draw_and_a_test():
    base = bench.walk_roofline([_level(4, 0, 4)], 1.0, {"sm_mhz": 1000.0}, {}, 1.0, num_sms=152)
    more = bench.walk_roofline([_level(8, 0, 8)], 1.0, {"sm_mhz": 1000.0}, {}, 1.0, num_sms=152)
    per_still = (more["achieved"] - base["achieved"]) * 1e9 / 4
    assert per_still == pytest.approx(42 / 4 + 2 + 1, rel=1e-12)


def test_fp64_judge_agrees_with_the_oracle_taylor():
    # bench.py states every error against scipy's expm_multiply; on the
    # metric's graph (smaller) and with a source term it must agree with the
    # oracle's FP64 Taylor values to rounding
    import numpy as np
    import mlmc_inputs as I
    from oracle import reference as R
    b = I.ba_graph(3000, 4, seed=5)
    t = 1.0 / I.lambda_max(b)
    v = np.ones(b.n)
    x = bench._fp64_judge(b, t, v)
    ref = R.expmv_taylor(b.scipy(), t, v)
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)
    a = I.convdiff_3d(8)
    t = 8.0 / float(abs(a.scipy()).sum(axis=1).max())
    v = np.random.default_rng(2).random(a.n)
    f = np.ones(a.n)
    u = bench._fp64_judge(a, t, v, f)
    ref = R.expmv_taylor(a.scipy(), t, v) + R.expmv_source_taylor(a.scipy(), t, f)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)
