"""The FP32 walk decides whether a walk ever leaves its start row by comparing
the index of its first uniform (a word of the block shared by four walks)
with a per-row threshold index instead of evaluating -ln(u).  These tests put one walk's first draw exactly on that
threshold (from either side) by choosing t, and check the GPU trajectory and
value against the oracle, which evaluates the holding time directly."""
import numpy as np
import pytest
import scipy.sparse as sp

import mlmc_inputs as I
from oracle import walker as W

from gpu_helpers import compare_walks, gpu_trace, make_plan, oracle_walks

pytestmark = pytest.mark.gpu

SEED, LEVEL = 12345, 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _first_draw_index(seed, row, rep, level):
    # FP32 rows with 1/(tL) >= 1: the first uniform is word (rep mod 4) of
    # the block of group rep // 4 (draw index 0xFFFFFFFE)
    g = rep >> 2
    x = W.philox([g & 0xFFFFFFFF, row, 0xFFFFFFFE, level | ((g >> 32) << 8)],
                 [seed & 0xFFFFFFFF, seed >> 32])
    return int(x[rep & 3]) >> 9


def _u(i):
    return np.float32((2.0 * i + 1.0) * 2.0 ** -24)


def _rate_at_boundary(i, side):
    """An FP32 factor ir = 1/(t L) with fl(-ln(u_i) ir) >= 1 and
    fl(-ln(u_{i+1}) ir) < 1 (side 'still': walk i just never jumps), or with
    fl(-ln(u_i) ir) < 1 and fl(-ln(u_{i-1}) ir) >= 1 (side 'jump')."""
    h = {k: np.float32(W.neglog32(np.array([_u(k)], np.float32))[0]) for k in (i - 1, i, i + 1)}
    ir = np.float32(1.0) / h[i]
    while np.float32(h[i] * ir) >= 1:
        ir = np.nextafter(ir, np.float32(0))
    below = ir                           # largest with fl(h_i ir) < 1
    above = np.nextafter(ir, np.float32(np.inf))  # smallest with fl(h_i ir) >= 1
    if side == "still":
        assert np.float32(h[i] * above) >= 1
        return above if np.float32(h[i + 1] * above) < 1 else None
    assert np.float32(h[i] * below) < 1
    return below if np.float32(h[i - 1] * below) >= 1 else None


@pytest.mark.parametrize("side", ["still", "jump"])
def test_first_draw_on_the_threshold(side):
    # rows 0 and 1 of [[0, 1], [1, 0]] (plus a pendant pair) have L = 1, so
    # the table's FP32 factor is fl(1/t) = ir for t = 1/ir
    a = I.to_csr(sp.csr_matrix(np.array([[0.0, 1.0, 0.0, 0.0], [1.0, 0.0, 0.0, 0.0],
                                         [0.0, 0.0, -0.5, 2.0], [0.0, 0.0, 3.0, 0.0]])))
    v = np.array([1.0, -2.0, 0.5, 3.0])
    for rep in range(64):
        i = _first_draw_index(SEED, 0, rep, LEVEL)
        ir = _rate_at_boundary(i, side)
        if ir is not None:
            break
    assert ir is not None
    t = 1.0 / float(ir)
    tb = W.build_tables(a, t)
    assert tb.inv_rate32[0] == ir
    reps = 64
    with make_plan(a, t, 1) as plan:
        assert plan.export_tables()["inv_rate32"][0] == ir
        got = gpu_trace(plan, LEVEL, False, 0, reps, v, seed=SEED)
    rows = np.repeat(np.arange(a.n), reps)
    rr = np.tile(np.arange(reps), a.n)
    orc, wk = oracle_walks(a, t, v, SEED, False, rows, rr, LEVEL, False)
    compare_walks(got, orc, v, wk.tables.dl, LEVEL, False, f"threshold/{side}")
    # the boundary walk: row 0, replica `rep`
    assert got["jumps"][rep] == (0 if side == "still" else orc["jumps"][rep])
    assert (orc["jumps"][rep] == 0) == (side == "still")
