"""The L2 access-policy window of the walk kernels (schedule l2_persist):
reported window sizes, and walks that are the same with and without it."""
import numpy as np
import pytest

import mlmc_inputs as I

from gpu_helpers import gpu_trace, make_plan, small_problems

pytestmark = pytest.mark.gpu

PROBLEMS = small_problems()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("prec", [0, 1])
def test_window_covers_the_tables(prec):
    a, t, v = PROBLEMS["ba_3001"]
    with make_plan(a, t, prec, l2_persist=1) as plan:
        w = plan.l2_window()
    with make_plan(a, t, prec, l2_persist=0) as plan:
        assert plan.l2_window() == {"bytes": 0, "hit_ratio": 0.0}
    assert w["bytes"] > 0          # GB300: persisting L2 and access-policy windows
    row, entry = (16, 48) if prec == 1 else (32, 80)   # row record, fused alias entry
    assert w["bytes"] >= row * a.n + entry * a.nnz
    assert w["bytes"] < row * a.n + entry * a.nnz + 1024
    assert w["hit_ratio"] == 1.0


def test_window_larger_than_the_set_aside_has_partial_hit_ratio():
    # ~2.2e6 fused entries of 48 B: ~110 MB of FP32 tables, above GB300's
    # persisting set-aside (about 85 MB) and below its 128 MB window limit
    a = I.ba_graph(140_000, 8, seed=3)
    with make_plan(a, 0.01, 1, l2_persist=1) as plan:
        w = plan.l2_window()
    assert 100e6 < w["bytes"] < 128 * 2 ** 20
    assert 0.5 < w["hit_ratio"] < 1.0


@pytest.mark.parametrize("prec", [0, 1])
def test_walks_are_the_same_with_and_without_the_window(prec):
    a, t, v = PROBLEMS["signed_301"]
    recs = []
    for flag in (1, 0):
        with make_plan(a, t, prec, l2_persist=flag) as plan:
            recs.append(gpu_trace(plan, 4, True, 0, 64, v, seed=99))
    assert np.array_equal(recs[0], recs[1])
