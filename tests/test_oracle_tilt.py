"""Pins of the oracle's walk with tilted clocks (the h-transform proposal).

The walk keeps the paper's structure (Algorithm 2: exponential holding
times, alias jumps, the Strang weights of Eq. 2 on the level grid) with
other rates lambda and jump law q, and a likelihood-ratio factor per jump.
What is pinned here, against things other than the code under test:
  - the general exact-moment recursion reduces to the paper's walk for
    lambda = L, q = k (the plain recursion is pinned elsewhere by brute force);
  - its mean equals the Strang product of the tilted split computed by an
    independent route (sparse Taylor / Pade of the split, not the kernels);
  - with h the Perron vector of a symmetric nonnegative A the tilted split's
    diagonal is constant (lambda_max I), so the Strang product is exp(tA)v
    exactly at every level: a closed form;
  - the C walker's tilted tables (rates, dl, log-ratios) reproduce the FP64
    law, and its walks match the exact first and second moments (z-tests);
  - the variance the clock tilt removes: on Barabasi-Albert graphs with h
    the exact solution the total relative variance stays near 0.13 while the
    paper's walk's grows with the hubs (0.53 at n = 500, 2.7 at n = 2000);
    with h = sqrt(x v), the geometric mean of the start value x and the end
    value v of the zero-variance h(s) = exp((1-s)tA)v, it is below 0.01 at
    level 0 (one Strang step);
  - beyond level 0 the exponent moves: from level 3 on, h = x^(3/4) v^(1/4)
    gives the smallest exact variance of the three forms x^a v^(1-a),
    a = 1/2, 3/4, 1 (0.068 against 0.094 and 0.130 at n = 500, level 7).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W


def _signed(n=9, seed=4):
    a = I.random_sparse(n, 3, seed=seed, signed=True, diag=True)
    return a, a.dense()


def _h(n, seed, spread=2.0):
    rng = np.random.default_rng(seed)
    return np.exp(spread * rng.standard_normal(n)).astype(np.float32)


def _h_clamped(ad, seed):
    # a positive h whose rates hit both clamps: one row far above its
    # neighbours (lambda below L/1024) and one far below (lambda above 4 L)
    n = ad.shape[0]
    h = _h(n, seed, spread=0.5)
    off = np.abs(ad.copy())
    np.fill_diagonal(off, 0.0)
    rows = np.flatnonzero(off.sum(axis=1) > 0)
    h[rows[0]] = 1e5
    h[rows[-1]] = 1e-5
    return h


@pytest.mark.parametrize("level,coarse", [(0, False), (2, False), (3, True)])
def test_general_moments_reduce_to_the_papers_walk(level, coarse):
    a, ad = _signed()
    t = 0.7
    v = np.random.default_rng(1).standard_normal(a.n)
    off = np.abs(ad.copy())
    np.fill_diagonal(off, 0.0)
    lii = off.sum(axis=1)
    q = np.where(lii[:, None] > 0, off / np.where(lii > 0, lii, 1.0)[:, None], 0.0)
    m1, m2 = R.level_moments(ad, t, v, level, coarse)
    g1, g2 = R.level_moments(ad, t, v, level, coarse, lam=lii, q=q)
    assert np.allclose(g1, m1, rtol=1e-12, atol=1e-14)
    assert np.allclose(g2, m2, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("level", [0, 1, 3])
def test_tilted_mean_is_the_tilted_strang_product(level):
    # the mean of the tilted walk (kernels exp(dt G1)) against the Strang
    # product of the split D' = diag(a_ii + lam), T' = diag(lam) - N applied
    # step by step (e^{dt D'/2} e^{-dt T'} e^{dt D'/2})^N v
    a, ad = _signed(12, 9)
    t = 0.9
    v = np.random.default_rng(2).standard_normal(a.n)
    lam, q = R.tilt_law(ad, _h_clamped(ad, 3), 0.2, t)   # both clamps active
    m1, _ = R.level_moments(ad, t, v, level, False, lam=lam, q=q)
    xs = R.strang(a.scipy(), t, v, level, lam=lam)
    assert np.allclose(m1, xs, rtol=1e-11, atol=1e-13)


def test_clamps_of_the_rates_are_active_in_the_pins():
    a, ad = _signed(12, 9)
    t = 0.9
    lam, _ = R.tilt_law(ad, _h_clamped(ad, 3), 0.2, t)
    off = np.abs(ad.copy())
    np.fill_diagonal(off, 0.0)
    lii = off.sum(axis=1)
    rows = lii > 0
    assert np.any(np.isclose(lam[rows], lii[rows] / 1024.0))
    assert np.any(np.isclose(lam[rows], np.maximum(lii[rows], 2.0 / t)))


@pytest.mark.parametrize("level", [0, 2, 4])
def test_perron_h_makes_the_split_exact(level):
    # symmetric nonnegative A, h = its Perron vector: lambda_i = (A h)_i / h_i
    # = lambda_max for every row (no clamp), D' = lambda_max I commutes with
    # T', and every level's Strang product is exp(tA) v
    b = I.ba_graph(60, 3, seed=2)
    ad = b.dense()
    w, vecs = np.linalg.eigh(ad)
    phi = np.abs(vecs[:, -1])
    t = 1.0 / w[-1]
    v = np.random.default_rng(5).random(b.n)
    lam, q = R.tilt_law(ad, phi, 0.0, t)
    assert np.allclose(lam, w[-1], rtol=1e-10)
    exact = sla.expm(t * ad) @ v
    assert np.allclose(R.strang(b.scipy(), t, v, level, lam=lam), exact, rtol=1e-11)
    m1, _ = R.level_moments(ad, t, v, level, False, lam=lam, q=q)
    assert np.allclose(m1, exact, rtol=1e-11)
    # the paper's split is not exact at this level
    assert not np.allclose(R.strang(b.scipy(), t, v, level), exact, rtol=1e-6)


def test_c_tables_reproduce_the_fp64_law():
    a, ad = _signed(40, 12)
    t = 0.6
    h = _h_clamped(ad, 8)
    tb = W.build_tables(a, t, h, 0.15, clocks=True)
    lam, q = R.tilt_law(ad, h.astype(np.float64), 0.15, t)
    assert np.allclose(tb.lam, lam, rtol=1e-14, atol=0)
    rows = lam > 0
    assert np.allclose(tb.inv_rate[rows], 1.0 / (t * lam[rows]), rtol=1e-15)
    assert np.allclose(tb.dl, t * (np.diag(ad) + lam), rtol=1e-14, atol=1e-15)
    # the kept column's log-ratio of every bucket: log(k/q) + log(L/lam)
    off = np.abs(ad.copy())
    np.fill_diagonal(off, 0.0)
    lii = off.sum(axis=1)
    for i in range(a.n):
        for b in range(tb.deg[i]):
            pos = a.row_ptr[i] + b
            j = tb.keep_col[pos]
            want = np.log((off[i, j] / lii[i]) / q[i, j]) + np.log(lii[i] / lam[i])
            assert abs(tb.lr_keep[pos] - want) <= 4 * np.spacing(np.float32(abs(want)) + 1e-30)
    # the jump law the tables sample is q (exact bucket law, as for the
    # proposal without tilted clocks)
    for i in range(a.n):
        k = tb.deg[i]
        if k == 0:
            continue
        got = {}
        for b in range(k):
            pos = a.row_ptr[i] + b
            keep = tb.thr[pos] / 2.0 ** 32
            got[tb.keep_col[pos]] = got.get(tb.keep_col[pos], 0.0) + keep / k
            got[tb.alias_col[pos]] = got.get(tb.alias_col[pos], 0.0) + (1.0 - keep) / k
        for j, p in got.items():
            assert abs(p - q[i, j]) <= k * 2.0 ** -31


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
@pytest.mark.parametrize("level,coarse", [(1, False), (3, True)])
def test_tilted_walks_match_exact_moments(precision, level, coarse):
    a = I.random_sparse(7, 3, seed=31, signed=True, diag=True)
    ad = a.dense()
    t = 0.8
    v = np.random.default_rng(2).random(7) - 0.4
    h = _h(a.n, 6, spread=1.0)
    lam, q = R.tilt_law(ad, h.astype(np.float64), 0.1, t)
    m1, m2 = R.level_moments(ad, t, v, level, coarse, lam=lam, q=q)
    reps = 1 << 16
    tb = W.build_tables(a, t, h, 0.1, clocks=True)
    wk = W.Walker(a, t, v, seed=77, precision=precision, tables=tb)
    rows = np.repeat(np.arange(a.n), reps)
    rr = np.tile(np.arange(reps), a.n)
    y = wk.walks(rows, rr, level, coarse)["y"].reshape(a.n, reps)
    var = m2 - m1 * m1
    noisy = var > 1e-12 * np.maximum(m2, 1e-300)
    # rows that cannot jump are deterministic: their samples are exact
    assert np.allclose(y[~noisy].mean(axis=1), m1[~noisy], rtol=1e-12, atol=1e-14)
    assert noisy.sum() >= 4
    z = (y[noisy].mean(axis=1) - m1[noisy]) / np.sqrt(var[noisy] / reps)
    assert np.all(np.abs(z) < 4.0), z
    # second moment: sample mean of y^2 against m2 (its standard error from
    # the sample fourth moment)
    y2 = y[noisy] * y[noisy]
    sv = y2.var(axis=1)
    seen = sv > 0
    z2 = (y2.mean(axis=1)[seen] - m2[noisy][seen]) / np.sqrt(sv[seen] / reps)
    assert np.all(np.abs(z2) < 4.5), z2
    # a row whose samples are all equal: its second moment comes from walks
    # too rare to appear among these (the mean is then within 4 sigma too)
    assert np.all(np.abs(y2.mean(axis=1)[~seen] - m2[noisy][~seen]) <= m2[noisy][~seen])


@pytest.mark.parametrize("n,plain_min", [(500, 0.4), (2000, 2.0)])
def test_clock_tilt_removes_the_hub_variance(n, plain_min):
    # Barabasi-Albert graph, beta = 1/lambda_max, v = 1 (total
    # communicability): the paper's walk's relative variance grows with the
    # hub degrees; the h-transform with h = exp(tA)1 keeps it near 0.13, and
    # tilting only the jumps (the clocks untouched) does not
    b = I.ba_graph(n, 4, seed=5)
    ad = b.dense()
    t = 1.0 / I.lambda_max(b)
    v = np.ones(n)
    x = sla.expm(t * ad) @ v
    lam, q = R.tilt_law(ad, x, 0.1, t)
    off = ad.copy()
    np.fill_diagonal(off, 0.0)
    lii = off.sum(axis=1)

    def relvar(lam_, q_):
        m1, m2 = R.level_moments(ad, t, v, 0, False, lam=lam_, q=q_)
        return (m2 - m1 * m1).sum() / (m1 * m1).sum()

    plain = relvar(None, None)
    jumps = relvar(lii, q)
    both = relvar(lam, q)
    assert plain > plain_min
    assert both < 0.2
    assert both < plain / 4 and both < jumps / 2
    lam_g, q_g = R.tilt_law(ad, np.sqrt(x * v), 0.1, t)
    assert relvar(lam_g, q_g) < 0.01


def test_three_quarter_power_tilt_is_best_beyond_level_0():
    # the same graph family: exact relative variance of the tilted walk with
    # h = x^a v^(1-a) at level 0 and at the levels the solver uses
    b = I.ba_graph(500, 4, seed=5)
    ad = b.dense()
    t = 1.0 / I.lambda_max(b)
    v = np.ones(b.n)
    x = sla.expm(t * ad) @ v

    def relvar(a, level):
        lam, q = R.tilt_law(ad, x ** a * v ** (1 - a), 0.1, t)
        m1, m2 = R.level_moments(ad, t, v, level, False, lam=lam, q=q)
        return (m2 - m1 * m1).sum() / (m1 * m1).sum()

    at0 = [relvar(a, 0) for a in (0.5, 0.75, 1.0)]
    assert at0[0] == min(at0)                       # level 0: the square root
    for level in (3, 7):
        r = [relvar(a, level) for a in (0.5, 0.75, 1.0)]
        assert r[1] < 0.8 * r[0] and r[1] < 0.6 * r[2], (level, r)
