"""Pins for the oracle's source term (Algorithm 3, reading R17): the exact
integral int_0^t exp(sA) f ds, the level-l Simpson mean, and the walker's
per-walk Simpson sums.  Each is checked against something other than itself:
closed forms for diagonal A, convergence of the level mean to the exact
integral, and z-tests of the walks against the deterministic level means."""
import numpy as np
import pytest
import scipy.sparse as sp

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W


def _signed():
    a = I.random_sparse(30, 3, seed=21, signed=True, diag=True)
    rng = np.random.default_rng(5)
    return a, 0.7, rng.standard_normal(a.n), rng.standard_normal(a.n)


def test_exact_source_integral_for_diagonal_a():
    d = np.array([-2.0, -0.5, 0.0, 0.3, 1.1])
    f = np.array([1.0, -2.0, 0.5, 3.0, -1.0])
    t = 0.8
    got = R.expmv_source_exact(sp.diags(d).tocsr(), t, f)
    want = np.where(d != 0, f * np.expm1(t * d) / np.where(d != 0, d, 1.0), t * f)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-15)


def test_exact_source_integral_matches_quadrature_of_exp():
    # int_0^t e^{sA} f ds by a fine composite Gauss-Legendre rule on e^{sA} f
    a, t, _, f = _signed()
    x, w = np.polynomial.legendre.leggauss(12)
    tot = np.zeros(a.n)
    panels = 16
    for p in range(panels):
        lo, hi = p * t / panels, (p + 1) * t / panels
        for xi, wi in zip(x, w):
            s = 0.5 * (hi - lo) * xi + 0.5 * (hi + lo)
            tot += 0.5 * (hi - lo) * wi * R.expmv(a.scipy(), s, f)
    assert np.allclose(R.expmv_source_exact(a.scipy(), t, f), tot, rtol=1e-11, atol=1e-13)


def test_level_mean_for_diagonal_a_is_simpson_of_the_exponential():
    d = np.array([-1.5, 0.4, 0.0])
    f = np.array([2.0, -1.0, 0.5])
    t = 1.2
    for level in (1, 3):
        n = 1 << level
        h = t / n
        w = np.array([1.0] + [4.0 if k % 2 else 2.0 for k in range(1, n)] + [1.0])
        want = (h / 3.0) * sum(w[k] * np.exp(k * h * d) * f for k in range(n + 1))
        got = R.strang_source(sp.diags(d).tocsr(), t, f, level)
        assert np.allclose(got, want, rtol=1e-13, atol=0)
        if level >= 2:
            hc = 2 * h
            wc = np.array([1.0] + [4.0 if k % 2 else 2.0 for k in range(1, n // 2)] + [1.0])
            want_c = (hc / 3.0) * sum(wc[k] * np.exp(k * hc * d) * f for k in range(n // 2 + 1))
            assert np.allclose(R.strang_source(sp.diags(d).tocsr(), t, f, level, coarse=True),
                               want_c, rtol=1e-13, atol=0)


def test_level_mean_converges_at_second_order():
    a, t, _, f = _signed()
    exact = R.expmv_source_exact(a.scipy(), t, f)
    errs = [np.linalg.norm(R.strang_source(a.scipy(), t, f, l) - exact) for l in range(3, 8)]
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.3), ratios


def test_source_part_of_a_walk_that_never_jumps():
    # diagonal A: every walk stays at its row, so its source part is the
    # Simpson sum of f_i e^{s d_i} exactly
    d = np.linspace(-1.0, 0.5, 8)
    a = I.to_csr(sp.diags(d).tocsr())
    f = np.random.default_rng(2).standard_normal(8)
    t, level = 0.9, 3
    wk = W.Walker(a, t, np.ones(8), seed=4, f=f)
    rec = wk.walks(np.arange(8), np.zeros(8, np.int64), level, False)
    want = R.strang_source(sp.diags(d).tocsr(), t, f, level)
    assert np.allclose(rec["src"], want, rtol=1e-13, atol=0)
    rec_c = wk.walks(np.arange(8), np.zeros(8, np.int64), level, True)
    want_c = want - R.strang_source(sp.diags(d).tocsr(), t, f, level, coarse=True)
    assert np.allclose(rec_c["src"], want_c, rtol=1e-9, atol=1e-14)


def test_zero_source_gives_zero_source_part():
    a, t, v, _ = _signed()
    wk = W.Walker(a, t, v, seed=3, f=np.zeros(a.n))
    rec = wk.walks(np.arange(a.n), np.zeros(a.n, np.int64), 2, True)
    assert np.all(rec["src"] == 0.0)
    plain = W.Walker(a, t, v, seed=3).walks(np.arange(a.n), np.zeros(a.n, np.int64), 2, True)
    assert np.array_equal(rec["y"], plain["y"]) and np.array_equal(rec["hash"], plain["hash"])


@pytest.mark.parametrize("level,coarse", [(1, False), (3, False), (3, True)])
def test_walk_source_means_match_level_means(level, coarse):
    a, t, v, f = _signed()
    want = R.strang_source(a.scipy(), t, f, level)
    if coarse:
        want = want - R.strang_source(a.scipy(), t, f, level, coarse=True)
    wk = W.Walker(a, t, np.zeros(a.n), seed=10 + level, f=f)
    m = 4000
    rows = np.repeat(np.arange(a.n), m)
    reps = np.tile(np.arange(m), a.n)
    rec = wk.walks(rows, reps, level, coarse)
    s = rec["src"].reshape(a.n, m)
    mean = s.mean(axis=1)
    se = s.std(axis=1, ddof=1) / np.sqrt(m)
    ok = se > 1e-12 * np.abs(want).max()       # rows without off-diagonals are deterministic
    z = (mean - want)[ok] / se[ok]
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    assert np.all(np.abs(mean - want)[~ok] <= 1e-12 * np.abs(want).max())


def test_mlmcl_sums_both_parts():
    a, t, v, f = _signed()
    wk = W.Walker(a, t, v, seed=8, f=f)
    sy, _, _, _ = wk.mlmcl(2, True, 0, 50)
    rows = np.repeat(np.arange(a.n), 50)
    rec = wk.walks(rows, np.tile(np.arange(50), a.n), 2, True)
    want = (rec["y"] + rec["src"]).reshape(a.n, 50).sum(axis=1)
    assert np.allclose(sy, want, rtol=1e-12, atol=1e-14)


def test_sparse_augmented_taylor_matches_dense_integral():
    a, t, _, f = _signed()
    assert np.allclose(R.expmv_source_taylor(a.scipy(), t, f),
                       R.expmv_source_exact(a.scipy(), t, f), rtol=1e-12, atol=1e-14)
