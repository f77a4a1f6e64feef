"""Pins of the oracle's walk with a proposal that changes with time (reading
R19: K equal pieces of scaled time, each with its own tilted rates, jump law
and d_i; a pending holding time carried over a piece boundary at the new
rate; each grid interval's own piece at both of its ends).

What is pinned here, against things other than the code under test:
  - one piece is the static tilted law: the same exact moments and the same
    tables;
  - the exact level means converge to exp(tA)v (scipy's expm) at weak order
    2 with four pieces of different laws, so the boundary rule (the mean of
    the two pieces at a boundary point) keeps the paper's order; a one-sided
    rule would be first order;
  - the C walker's walks match the exact first and second moments (z-tests),
    FP64 and FP32, fine and coupled levels, and the fraction of walks that
    never jump matches exp(-t * integral of lambda) (the carried-over holding
    time is the inhomogeneous exponential clock);
  - its pair form (Eq. 7) equals its running products of Algorithm 2;
  - the variance the time pieces remove on a Barabasi-Albert graph: h_p =
    T3((1 - s_p) t |A|) |v| at the middle s_p of each piece (the Taylor
    approximation of the zero-variance h(s) = exp((1-s)tA)v) against the best
    static form x^(3/4) v^(1/4).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W


def _hs(n, k, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    return np.exp(spread * rng.standard_normal((k, n))).astype(np.float32)


def _laws(ad, t, hs, alpha=0.1):
    return [R.tilt_law(ad, h.astype(np.float64), alpha, t) for h in hs]


def _taylor_h(ad, t, v, s, terms=3):
    out = np.abs(v).astype(np.float64)
    term = out.copy()
    for k in range(1, terms + 1):
        term = (s * t) * (np.abs(ad) @ term) / k
        out = out + term
    return out


@pytest.mark.parametrize("level,coarse", [(2, False), (3, True)])
def test_one_piece_is_the_static_law(level, coarse):
    a = I.random_sparse(9, 3, seed=4, signed=True, diag=True)
    ad = a.dense()
    t = 0.7
    v = np.random.default_rng(1).random(9) - 0.3
    h = _hs(a.n, 1, 3)
    lam, q = R.tilt_law(ad, h[0].astype(np.float64), 0.1, t)
    m1, m2 = R.level_moments(ad, t, v, level, coarse, lam=lam, q=q)
    p1, p2 = R.level_moments_pieces(ad, t, v, level, coarse, [(lam, q)])
    assert np.array_equal(m1, p1) and np.array_equal(m2, p2)
    tb = W.build_tables_pieces(a, t, h, 0.1)
    ref = W.build_tables(a, t, h[0], 0.1, clocks=True)
    assert tb.pieces == 1
    for name in ("thr", "keep_col", "alias_col", "lr_keep", "lr_alias", "inv_rate32", "dl"):
        assert np.array_equal(getattr(tb, name), getattr(ref, name)), name


def test_piece_boundaries_keep_weak_order_two():
    a = I.random_sparse(12, 3, seed=8, signed=True, diag=True)
    ad = a.dense()
    t = 0.9
    v = np.random.default_rng(5).random(12) + 0.2
    x = sla.expm(t * ad) @ v
    laws = _laws(ad, t, _hs(a.n, 4, 11, spread=1.5))
    errs = []
    for level in range(2, 8):
        m1, _ = R.level_moments_pieces(ad, t, v, level, False, laws)
        errs.append(np.linalg.norm(m1 - x) / np.linalg.norm(x))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.7) & (ratios < 4.3)), ratios


def test_pieces_need_every_boundary_on_the_grid():
    a = I.random_sparse(6, 2, seed=2, signed=False, diag=True)
    ad = a.dense()
    hs = _hs(a.n, 4, 1)
    with pytest.raises(ValueError):
        R.level_moments_pieces(ad, 0.5, np.ones(6), 1, False, _laws(ad, 0.5, hs))
    wk = W.Walker(a, 0.5, np.ones(6), seed=1, tables=W.build_tables_pieces(a, 0.5, hs, 0.1))
    assert wk.walk(0, 0, 1, False).status == -1   # N = 2 intervals, 4 pieces
    assert wk.walk(0, 0, 2, False).status == 0


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
@pytest.mark.parametrize("level,coarse,k", [(2, False, 4), (3, True, 2), (3, True, 4)])
def test_piece_walks_match_exact_moments(precision, level, coarse, k):
    a = I.random_sparse(7, 3, seed=31, signed=True, diag=True)
    ad = a.dense()
    t = 0.8
    v = np.random.default_rng(2).random(7) - 0.4
    hs = _hs(a.n, k, 6 + k)
    m1, m2 = R.level_moments_pieces(ad, t, v, level, coarse, _laws(ad, t, hs))
    reps = 1 << 16
    wk = W.Walker(a, t, v, seed=77, precision=precision, tables=W.build_tables_pieces(a, t, hs, 0.1))
    rows = np.repeat(np.arange(a.n), reps)
    rr = np.tile(np.arange(reps), a.n)
    rec = wk.walks(rows, rr, level, coarse)
    assert np.all(rec["status"] == 0)
    y = rec["y"].reshape(a.n, reps)
    var = m2 - m1 * m1
    noisy = var > 1e-12 * np.maximum(m2, 1e-300)
    assert np.allclose(y[~noisy].mean(axis=1), m1[~noisy], rtol=1e-12, atol=1e-14)
    assert noisy.sum() >= 4
    z = (y[noisy].mean(axis=1) - m1[noisy]) / np.sqrt(var[noisy] / reps)
    assert np.all(np.abs(z) < 4.0), z
    y2 = y[noisy] * y[noisy]
    sv = y2.var(axis=1)
    seen = sv > 0
    z2 = (y2.mean(axis=1)[seen] - m2[noisy][seen]) / np.sqrt(sv[seen] / reps)
    assert np.all(np.abs(z2) < 4.5), z2
    # Eq. 7's pair form against Algorithm 2's running products, walk by walk
    scale = np.abs(rec["y"]).max()
    assert np.max(np.abs(rec["y"] - rec["y_alg2"])) <= 1e-12 * scale


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_carried_holding_time_is_the_inhomogeneous_clock(precision):
    # P(no jump on [0, 1]) = exp(-t sum_p lambda_p / K) for each start row:
    # a wrong carry-over (the quotient inverted, the residual dropped or
    # redrawn from the boundary) changes it
    a = I.random_sparse(8, 3, seed=12, signed=False, diag=True)
    ad = a.dense()
    t = 0.6
    k = 4
    hs = _hs(a.n, k, 21, spread=1.2)
    lam = np.array([lq[0] for lq in _laws(ad, t, hs)])       # [K, n]
    p_still = np.exp(-t * lam.mean(axis=0))
    reps = 1 << 16
    wk = W.Walker(a, t, np.ones(a.n), seed=5, precision=precision,
                  tables=W.build_tables_pieces(a, t, hs, 0.1))
    rows = np.repeat(np.arange(a.n), reps)
    rr = np.tile(np.arange(reps), a.n)
    still = (wk.walks(rows, rr, 2, False)["jumps"].reshape(a.n, reps) == 0).mean(axis=1)
    z = (still - p_still) / np.sqrt(p_still * (1 - p_still) / reps)
    assert np.all(np.abs(z) < 4.0), (z, still, p_still)
    # the clocks differ enough between pieces for the test to see a carry-over
    assert np.max(lam.max(axis=0) / lam.min(axis=0)) > 2.0


def test_time_pieces_cut_the_variance_on_ba_graphs():
    b = I.ba_graph(300, 4, seed=5)
    ad = b.dense()
    t = 1.0 / I.lambda_max(b)
    v = np.ones(b.n)
    x = sla.expm(t * ad) @ v

    def relvar(laws, level):
        m1, m2 = R.level_moments_pieces(ad, t, v, level, False, laws)
        return (m2 - m1 * m1).sum() / (m1 * m1).sum()

    static = [R.tilt_law(ad, x ** 0.75, 0.1, t)]
    for level in (3, 5):
        base = relvar(static, level)
        got = {}
        for k in (2, 4):
            hs = [_taylor_h(ad, t, v, 1.0 - (p + 0.5) / k) for p in range(k)]
            got[k] = relvar(_laws(ad, t, hs), level)
        assert got[2] < base / 2.5 and got[4] < base / 8.0, (level, base, got)


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_rows_without_off_diagonals_keep_their_walks(precision):
    # a row with no off-diagonal entries has rate 0 in every piece (inverse
    # rate infinite): its walks never jump, the carry-over keeps their
    # pending time infinite, and the sample is v_i e^{t a_ii} exactly; the
    # other rows still match the exact moments
    import scipy.sparse as sp
    base = I.random_sparse(8, 3, seed=14, signed=True, diag=True).dense()
    base[3, :] = 0.0
    base[3, 3] = -0.7
    a = I.to_csr(sp.csr_matrix(base))
    ad = a.dense()
    t = 0.6
    v = np.random.default_rng(4).random(8) + 0.1
    hs = _hs(a.n, 4, 5)
    m1, _ = R.level_moments_pieces(ad, t, v, 2, False, _laws(ad, t, hs))
    tb = W.build_tables_pieces(a, t, hs, 0.1)
    assert np.all(np.isinf(tb.inv_rate.reshape(4, a.n)[:, 3]))
    reps = 1 << 15
    wk = W.Walker(a, t, v, seed=9, precision=precision, tables=tb)
    rec = wk.walks(np.repeat(np.arange(a.n), reps), np.tile(np.arange(reps), a.n), 2, False)
    assert np.all(rec["status"] == 0)
    y = rec["y"].reshape(a.n, reps)
    jumps = rec["jumps"].reshape(a.n, reps)
    assert np.all(jumps[3] == 0)
    assert np.allclose(y[3], v[3] * np.exp(-0.7 * t), rtol=1e-12 if precision == W.FP64 else 1e-6)
    assert abs(m1[3] - v[3] * np.exp(-0.7 * t)) <= 1e-12 * v[3]
    others = [i for i in range(a.n) if i != 3]
    sd = y[others].std(axis=1) / np.sqrt(reps)
    z = (y[others].mean(axis=1) - m1[others]) / np.maximum(sd, 1e-300)
    assert np.all(np.abs(z) < 4.5), z
