"""Pins for the oracle walker: split and alias tables against their
definitions, and the walk's statistics against the exact moments."""
import numpy as np
import pytest
import scipy.sparse as sp

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W


def _exact_jump_law(tb, i):
    """Probability of each column under row i's alias table (exact in the
    threshold quantisation): bucket b w.p. 1/deg, keep w.p. thr/2^32."""
    k = int(tb.deg[i])
    p = {}
    for b in range(k):
        pos = int(tb.row_ptr[i]) + b
        keep = float(tb.thr[pos]) / 2.0 ** 32
        for c, w in ((int(tb.keep_col[pos]), keep), (int(tb.alias_col[pos]), 1.0 - keep)):
            p[c] = p.get(c, 0.0) + w / k
    return p


def test_split_quantities_match_definition():
    a = I.random_sparse(80, 5, seed=1, signed=True, diag=True)
    tb = W.build_tables(a, 0.37)
    d, lii, _, _ = R.split(a.dense())
    assert np.allclose(tb.L, lii, rtol=1e-15, atol=0)
    assert np.allclose(tb.dl, 0.37 * d, rtol=1e-15, atol=1e-300)
    assert np.array_equal(tb.deg, np.count_nonzero(a.dense() - np.diag(np.diag(a.dense())), 1))


def test_alias_tables_reproduce_jump_law():
    # Eq. 12: from row i the walk jumps to j with probability |a_ij|/L_ii and
    # picks up the sign of a_ij.
    a = I.random_sparse(60, 6, seed=2, signed=True, diag=True)
    tb = W.build_tables(a, 1.0)
    dense = a.dense()
    for i in range(a.n):
        if tb.deg[i] == 0:
            continue
        law = _exact_jump_law(tb, i)
        for j in range(a.n):
            if j == i:
                continue
            want = abs(dense[i, j]) / tb.L[i]
            assert abs(law.get(j, 0.0) - want) <= 1e-8
        for b in range(int(tb.deg[i])):
            pos = int(tb.row_ptr[i]) + b
            for c, neg in ((tb.keep_col[pos], tb.keep_neg[pos]),
                           (tb.alias_col[pos], tb.alias_neg[pos])):
                assert bool(neg) == (dense[i, c] < 0)


def test_alias_uniform_rows_always_keep():
    a = I.ba_graph(300, 3, seed=3)
    tb = W.build_tables(a, 0.1)
    assert np.all(tb.thr[: a.nnz] == 0xFFFFFFFF)
    assert np.array_equal(tb.keep_col[: a.nnz], tb.alias_col[: a.nnz])


def test_alias_hub_row_and_explicit_zeros():
    # a hub row of 2000 unequal weights plus rows with stored zeros
    rng = np.random.default_rng(5)
    n = 2001
    r = np.concatenate([np.zeros(n - 1, int), [5, 5, 7]])
    c = np.concatenate([np.arange(1, n), [6, 8, 9]])
    v = np.concatenate([rng.uniform(0.01, 3.0, n - 1), [0.0, 2.0, 0.0]])
    m = sp.csr_matrix((v, (r, c)), shape=(n, n))
    a = I.to_csr(m)
    a.val[a.row_ptr[7]:a.row_ptr[8]] = 0.0  # row 7: only a stored zero -> L = 0
    tb = W.build_tables(a, 1.0)
    law = _exact_jump_law(tb, 0)
    dense0 = m.toarray()[0]
    assert max(abs(law.get(j, 0.0) - dense0[j] / dense0.sum()) for j in range(1, n)) <= 1e-8
    law5 = _exact_jump_law(tb, 5)
    assert abs(law5.get(8, 0.0) - 1.0) <= 1e-9 and law5.get(6, 0.0) <= 1e-9
    assert tb.L[7] == 0.0 and np.isinf(tb.inv_rate[7])


def _ztest(a, t, v, level, coarse, variant, precision=W.FP64, reps=100_000, seed=11):
    m1, m2 = R.level_moments(a.dense(), t, v, level, coarse)
    wk = W.Walker(a, t, v, seed=seed, precision=precision, variant=variant)
    s, s2, _, lim = wk.mlmcl(level, coarse, 0, reps)
    assert lim == 0
    sd = np.sqrt(np.maximum(m2 - m1 * m1, 0.0) / reps)
    z = (s / reps - m1) / np.where(sd > 0, sd, 1.0)
    # also returns the sample and exact total second moments (checked to 10%)
    return np.abs(z).max(), s2 / reps, m2.sum()


@pytest.mark.parametrize("variant", [W.RESIDUAL, W.REDRAW])
@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
@pytest.mark.parametrize("level,coarse", [(1, False), (2, True), (4, True)])
def test_walk_statistics_match_exact_moments(variant, precision, level, coarse):
    a = I.random_sparse(6, 2, seed=3, signed=True, diag=True)
    v = np.random.default_rng(5).random(6) - 0.3
    zmax, y2, m2 = _ztest(a, 0.7, v, level, coarse, variant, precision)
    assert zmax <= 4.0
    assert abs(y2 - m2) <= 0.1 * m2


def test_literal_old_rate_reading_is_rejected():
    # Reading R1: the listing draws S before choosing the new state; taken
    # literally, the holding time would use the old state's rate.  On a star
    # graph (hub degree 4, leaves 1) that reading misses the Strang mean by
    # many standard errors, while the CTMC reading matches it.
    a = I.star_graph(4)
    v = np.arange(1.0, 6.0)
    z_ok, _, _ = _ztest(a, 1.0, v, 2, False, W.RESIDUAL)
    z_bad, _, _ = _ztest(a, 1.0, v, 2, False, W.LITERAL_RATE)
    assert z_ok <= 4.0
    assert z_bad >= 10.0


def test_no_jump_walks_give_zero_correction():
    # Fig. 1 case (d): without a jump the fine and coarse weights agree.
    a = I.ring_graph(5)
    wk = W.Walker(a, 1e-6, np.arange(5.0), seed=3)
    recs = wk.walks(np.zeros(200, np.int64), np.arange(200), 3, True)
    nojump = recs[recs["jumps"] == 0]
    assert nojump.size > 150
    assert np.all(nojump["y"] == 0.0)


def test_diagonal_matrix_walks_are_deterministic():
    d = np.array([-1.0, 0.5, 2.0])
    a = I.to_csr(sp.diags(d))
    v = np.array([1.0, -2.0, 0.5])
    wk = W.Walker(a, 0.7, v, seed=1)
    for i in range(3):
        r = wk.walk(i, 17, 0, False)
        assert r.jumps == 0 and r.end == i
        assert abs(r.y - np.exp(0.7 * d[i]) * v[i]) <= 1e-15 * abs(r.y)
        r = wk.walk(i, 17, 4, True)
        assert r.y == 0.0


def test_stochastic_generator_weights_are_exactly_one():
    # A = Q with rows summing to zero and off-diagonals >= 0: d = 0 and no
    # sign flips, so every coarsest-level walk returns v_end = 1.
    a0 = I.random_sparse(40, 4, seed=6, signed=False, diag=False).scipy()
    q = I.to_csr(a0 - sp.diags(np.asarray(a0.sum(axis=1)).ravel()))
    wk = W.Walker(q, 1.5, np.ones(40), seed=2)
    s, s2, jumps, _ = wk.mlmcl(2, False, 0, 50)
    assert jumps > 0
    assert np.allclose(s, 50.0, rtol=0, atol=1e-12)


def test_paired_form_matches_algorithm2_products():
    a = I.random_sparse(30, 4, seed=8, signed=True, diag=True)
    v = np.random.default_rng(2).random(30)
    wk = W.Walker(a, 0.9, v, seed=4)
    recs = wk.walks(np.repeat(np.arange(30), 20), np.tile(np.arange(20), 30), 3, True)
    scale = np.exp(np.abs(recs["log_c"])) * np.abs(v[recs["end"]])
    assert np.all(np.abs(recs["y"] - recs["y_alg2"]) <= 1e-12 * scale)


def test_trajectories_are_counter_addressed():
    # Any walk can be replayed alone: walk (row, rep) does not depend on the
    # others, and different reps give different paths.
    a = I.random_sparse(40, 5, seed=9, signed=True, diag=True)
    wk = W.Walker(a, 2.0, np.ones(40), seed=99)
    row = int(np.argmax(wk.tables.deg))
    batch = wk.walks(np.full(64, row), np.arange(64), 2, True)
    single = wk.walk(row, 41, 2, True)
    assert batch[41]["hash"] == single.hash and batch[41]["end"] == single.end
    assert len(set(batch["hash"].tolist())) > 20


def test_walk_limit_is_reported():
    a = I.ring_graph(6)
    wk = W.Walker(a, 50.0, np.ones(6), seed=1, max_jumps=3)
    r = wk.walk(0, 0, 2, False)
    assert r.status == 1 and r.y == 0.0


# ---------------------------------------------------------------------------
# Importance-sampling proposal tables (the learned-proposal path)
# ---------------------------------------------------------------------------
def test_proposal_tables_sample_the_mixture_and_record_log_ratios():
    a = I.random_sparse(80, 6, seed=12, signed=True, diag=True)
    h = np.random.default_rng(4).uniform(0.2, 5.0, a.n).astype(np.float32)
    alpha = 0.15
    tb = W.build_tables(a, 0.7, h, alpha)
    dense = a.dense()
    for i in range(a.n):
        if tb.deg[i] == 0:
            continue
        off = [j for j in range(a.n) if j != i and dense[i, j] != 0.0]
        k = {j: abs(dense[i, j]) / tb.L[i] for j in off}
        hs = sum(abs(dense[i, j]) * float(h[j]) for j in off)
        q = {j: (1 - alpha) * abs(dense[i, j]) * float(h[j]) / hs + alpha * k[j] for j in off}
        law = _exact_jump_law(tb, i)
        assert max(abs(law.get(j, 0.0) - q[j]) for j in off) <= 1e-8
        for b in range(int(tb.deg[i])):
            pos = int(tb.row_ptr[i]) + b
            for c, lr in ((tb.keep_col[pos], tb.lr_keep[pos]), (tb.alias_col[pos], tb.lr_alias[pos])):
                assert abs(float(lr) - np.log(k[int(c)] / q[int(c)])) <= 1e-6 * (1 + abs(float(lr)))


@pytest.mark.parametrize("level,coarse", [(1, False), (3, True)])
def test_proposal_walks_are_unbiased(level, coarse):
    # E_q[Y prod k/q] equals the exact mean of the plain walk (Eq. 3, 8).
    a = I.random_sparse(6, 2, seed=3, signed=True, diag=True)
    v = np.random.default_rng(5).random(6) - 0.3
    h = np.random.default_rng(6).uniform(0.1, 10.0, 6).astype(np.float32)
    m1, m2 = R.level_moments(a.dense(), 0.7, v, level, coarse)
    tb = W.build_tables(a, 0.7, h, 0.2)
    wk = W.Walker(a, 0.7, v, seed=21, tables=tb)
    reps = 200_000
    s, s2, _, _ = wk.mlmcl(level, coarse, 0, reps)
    rows = m2 - m1 * m1 > 0
    # standard error from the proposal's own sample (its variance differs)
    per_row_var = np.maximum(s2 / reps / a.n, 1e-30)
    z = (s[rows] / reps - m1[rows]) / np.sqrt(np.maximum(m2[rows], per_row_var) / reps)
    assert np.abs(z).max() <= 4.0


def test_value_function_proposal_reduces_variance():
    # With h = x the jump choice follows the value of the next state (the
    # zero-variance importance-sampling idea); on a scale-free graph with
    # beta = 1/lambda_max the per-walk variance drops.
    a = I.ba_graph(500, 4, seed=3)
    t = 1.0 / I.lambda_max(a)
    v = np.ones(a.n)
    x = R.expmv(a.scipy(), t, v)
    m1, _ = R.level_moments(a.dense(), t, v, 3, False)

    def rel_var(tables):
        wk = W.Walker(a, t, v, seed=5, tables=tables)
        s, s2, _, _ = wk.mlmcl(3, False, 0, 4000)
        return (s2 - (s * s).sum() / 4000) / 3999 / (m1 ** 2).sum()

    plain = rel_var(W.build_tables(a, t))
    learned = rel_var(W.build_tables(a, t, x.astype(np.float32), 0.1))
    assert learned < 0.8 * plain


def test_fp32_first_uniform_comes_from_the_shared_block():
    # FP32 walks in rows with 1/(tL) >= 1 take their first uniform from word
    # (rep mod 4) of the block (rep // 4, row, 0xFFFFFFFE, level | rep_hi..);
    # the walk never jumps exactly when that uniform's holding time reaches 1.
    a = I.ring_graph(16)                     # L = 2 everywhere
    t = 0.3                                  # 1/(tL) = 1.67 >= 1
    seed, level = 99, 3
    wk = W.Walker(a, t, np.ones(a.n), seed=seed, precision=W.FP32)
    ir = wk.tables.inv_rate32
    assert ir[0] >= 1.0
    reps = np.arange(400)
    rows = np.zeros(reps.size, np.int64)
    rec = wk.walks(rows, reps, level, False)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    differ = 0
    for r, jumps in zip(reps, rec["jumps"]):
        xg = W.philox([r >> 2, 0, 0xFFFFFFFE, level], key)
        x0 = W.philox([r, 0, 0, level], key)
        def still(word):
            u = np.float32(((int(word) >> 8) | 1) * 2.0 ** -24)
            return np.float32(W.neglog32(np.array([u], np.float32))[0] * ir[0]) >= 1.0
        assert (jumps == 0) == still(xg[r & 3])
        differ += still(xg[r & 3]) != still(x0[0])
    assert differ > 20                       # the test tells the two layouts apart


def test_fp32_shared_block_keeps_the_still_probability():
    a = I.ring_graph(8)
    t = 0.4                                  # t L = 0.8: P(no jump) = e^-0.8
    wk = W.Walker(a, t, np.ones(a.n), seed=5, precision=W.FP32)
    m = 200000
    rec = wk.walks(np.zeros(m, np.int64), np.arange(m), 2, False)
    p = np.exp(-0.8)
    frac = (rec["jumps"] == 0).mean()
    assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / m)


def _hold_count(words_after_jump, first_word, ir):
    """Jumps of a walk with constant rate: the number of partial sums of
    FP32 holding times below 1, the first from `first_word`, the one after
    jump k from words_after_jump(k) (k = 0, 1, ...)."""
    def hold(word):
        u = np.float32(((int(word) >> 8) | 1) * 2.0 ** -24)
        return np.float32(W.neglog32(np.array([u], np.float32))[0] * ir)
    s = hold(first_word)
    jumps = 0
    while s < np.float32(1.0):
        s = np.float32(s + hold(words_after_jump(jumps)))
        jumps += 1
    return jumps


@pytest.mark.parametrize("t", [0.3, 1.4])
def test_fp32_holding_time_after_a_jump_comes_from_the_jump_draw(t):
    # FP32 walks: jump k + 1 takes words 2, 3 of draw k and the holding
    # time after it word 0 of the same draw; the first holding time takes
    # word 1 of draw 0 (rows with 1/(tL) < 1, t = 1.4) or the shared block
    # word (1/(tL) >= 1, t = 0.3).  On a ring every state has L = 2, so the
    # jump count depends on the holding-time words alone.
    a = I.ring_graph(16)
    seed, level, row = 12345, 4, 3
    wk = W.Walker(a, t, np.ones(a.n), seed=seed, precision=W.FP32)
    ir = wk.tables.inv_rate32[row]
    grouped = ir >= 1.0
    key = [seed & 0xFFFFFFFF, seed >> 32]
    reps = np.arange(300)
    rec = wk.walks(np.full(reps.size, row, np.int64), reps, level, False)
    old_layout_differs = 0
    for r, jumps in zip(reps, rec["jumps"]):
        draw = lambda k, r=r: W.philox([r, row, k, level], key)
        first = (W.philox([r >> 2, row, 0xFFFFFFFE, level], key)[r & 3] if grouped
                 else draw(0)[1])
        assert jumps == _hold_count(lambda k: draw(k)[0], first, ir)
        old_first = first if grouped else draw(0)[0]
        old_layout_differs += jumps != _hold_count(lambda k: draw(k + 1)[0], old_first, ir)
    assert rec["jumps"].max() >= 2
    assert old_layout_differs > 20           # the test tells the layouts apart


def test_fp32_forward_walk_uses_the_packed_layout():
    # Forward walk g: counter (g lo, g hi, draw, level | 1 << 6); its first
    # holding time is word 1 of draw 0, the one after jump k word 0 of draw k.
    a = I.ring_graph(12)
    t, seed, level = 1.2, 77, 3
    fw = W.ForwardWalker(a, t, np.ones(a.n), seed=seed, precision=W.FP32)
    ir = fw.tables.inv_rate32[0]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rec = fw.walks_fwd(0, 200, level, False)
    for g, jumps in enumerate(rec["jumps"]):
        draw = lambda k, g=g: W.philox([g, 0, k, level | (1 << 6)], key)
        assert jumps == _hold_count(lambda k: draw(k)[0], draw(0)[1], ir)
