"""Pins for the oracle's deterministic FP64 references (exp(tA)v, Strang
levels, exact moments) against closed forms, an independent library and
invariants."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import mlmc_inputs as I
from oracle import reference as R


def test_pade13_matches_scipy_expm():
    rng = np.random.default_rng(0)
    for scale in (0.1, 1.0, 8.0, 40.0):
        m = rng.standard_normal((40, 40)) * scale / 6.0
        ref = sla.expm(m)
        assert np.abs(R.expm_pade13(m) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_pade13_diagonal_closed_form():
    d = np.linspace(-30, 5, 17)
    assert np.allclose(R.expm_pade13(np.diag(d)), np.diag(np.exp(d)), rtol=1e-13, atol=0)


def test_expmv_dense_and_taylor_match_dst_closed_form():
    w = I.workload_c1()
    g, h = w.extra["grid"], w.extra["h"]
    ref = R.dst_expmv_laplacian_2d(g, 1.0 / h ** 2, w.t, w.v)
    dense = R.expmv(w.a.scipy(), w.t, w.v)
    taylor = R.expmv_taylor(w.a.scipy(), w.t, w.v)
    assert np.abs(dense - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(taylor - ref).max() <= 1e-13 * np.abs(ref).max()


def test_taylor_matches_pade_on_signed_nonsymmetric_matrix():
    a = I.random_sparse(300, 4, seed=11, signed=True, diag=True, scale=2.0)
    v = np.random.default_rng(1).standard_normal(a.n)
    ref = R.expm_pade13(1.3 * a.dense()) @ v
    got = R.expmv_taylor(a.scipy(), 1.3, v)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_stochastic_generator_preserves_ones():
    # Q with nonnegative off-diagonals and zero row sums: exp(tQ) 1 = 1.
    a = I.random_sparse(200, 5, seed=4, signed=False, diag=False).scipy()
    q = a - sp.diags(np.asarray(a.sum(axis=1)).ravel())
    ones = np.ones(200)
    assert np.abs(R.expmv_taylor(q, 2.5, ones) - 1).max() <= 1e-13
    assert np.abs(R.expm_pade13(2.5 * q.toarray()) @ ones - 1).max() <= 1e-13


def test_split_reconstructs_matrix():
    a = I.random_sparse(50, 4, seed=7, signed=True, diag=True).dense()
    d, lii, t, sigma = R.split(a)
    rec = np.diag(d) - t
    off = ~np.eye(a.shape[0], dtype=bool)
    assert np.array_equal(rec[off], a[off])  # off-diagonals exact
    # diagonal: (a_ii + L_ii) - L_ii, two roundings
    assert np.all(np.abs(np.diag(rec) - np.diag(a)) <= 4 * np.finfo(float).eps * (lii + 1))
    assert np.array_equal(sigma[off], (a[off] < 0).astype(int))
    assert np.all(lii >= 0)
    # the unsigned generator -L has zero row sums
    off = np.abs(a - np.diag(np.diag(a)))
    assert np.abs((off - np.diag(lii)).sum(axis=1)).max() <= 1e-12


def test_strang_weak_order_two():
    # Eq. 13: the global splitting error falls ~4x per level.
    w = I.workload_c1()
    ref = R.expmv(w.a.scipy(), w.t, w.v)
    errs = [np.linalg.norm(R.strang(w.a.scipy(), w.t, w.v, l) - ref) for l in range(1, 6)]
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.6) & (ratios < 4.4))


def test_strang_exact_when_d_and_t_commute():
    # Ring graph: D = 2I commutes with T, so Eq. 2 is exact at every level.
    a = I.ring_graph(12)
    v = np.random.default_rng(3).random(12)
    ref = R.expmv(a.scipy(), 0.9, v)
    for l in (0, 1, 3):
        assert np.abs(R.strang(a.scipy(), 0.9, v, l) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_strang_exact_for_diagonal_matrix():
    d = np.array([-1.0, 0.5, 2.0, -3.0])
    a = sp.diags(d).tocsr()
    v = np.array([1.0, -2.0, 0.5, 3.0])
    for l in (0, 2):
        assert np.allclose(R.strang(a, 0.7, v, l), np.exp(0.7 * d) * v, rtol=1e-14, atol=0)


@pytest.mark.parametrize("level,coarse", [(0, False), (1, False), (1, True), (2, True)])
def test_moments_transfer_matrices_match_brute_force(level, coarse):
    a = I.random_sparse(5, 2, seed=21, signed=True, diag=True)
    v = np.random.default_rng(2).standard_normal(5)
    m1, m2 = R.level_moments(a.dense(), 0.8, v, level, coarse)
    b1, b2 = R.brute_moments(a.dense(), 0.8, v, level, coarse)
    assert np.abs(m1 - b1).max() <= 1e-13 * max(1.0, np.abs(b1).max())
    assert np.abs(m2 - b2).max() <= 1e-13 * max(1.0, np.abs(b2).max())


def test_moment_means_are_strang_corrections():
    a = I.random_sparse(7, 3, seed=5, signed=True, diag=True)
    v = np.random.default_rng(9).random(7)
    means = R.level_means(a.scipy(), 0.6, v, 1, 4)
    for l in range(1, 5):
        m1, _ = R.level_moments(a.dense(), 0.6, v, l, l > 1)
        assert np.abs(m1 - means[l]).max() <= 1e-13


def test_lemma2_variance_order():
    # Lemma 2: E[(P_l - P_{l-1})^2] = O(dt_l^2): the exact second moment of
    # the correction falls ~4x per level.
    a = I.star_graph(4)
    v = np.random.default_rng(4).random(5)
    m2s = [R.level_moments(a.dense(), 1.0, v, l, True)[1].sum() for l in range(3, 8)]
    ratios = np.array(m2s[:-1]) / np.array(m2s[1:])
    assert np.all((ratios > 3.5) & (ratios < 4.5))


def test_choose_l0_rule():
    # Eq. 16: l0 = log2(2 beta d_max), rounded up.
    assert R.choose_l0(np.array([8.0]), np.array([8.0]), 1.0 / 8.0) == 1
    assert R.choose_l0(np.array([0.0, -1.0]), np.array([2.0, 1.0]), 1.0) == 2
    assert R.choose_l0(np.array([0.0]), np.array([0.0]), 1.0) == 0
