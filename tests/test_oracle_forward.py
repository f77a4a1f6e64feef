"""Pins for the oracle's forward mode (the full-vector representation, Eq. 5):
walks on B = A^T from starts drawn in proportion to |v|, each adding its
weighted contribution to x at the walk's end state.

The forward Strang mean is checked against the dense level-0 formula and
second-order convergence to exp(tA)v; the walker against the exact start law,
closed forms (diagonal A, column-stochastic generators) and z-tests of its
level means and coupled corrections."""
import numpy as np
import pytest
import scipy.sparse as sp

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W


def _nonsym():
    a = I.random_sparse(40, 4, seed=8, signed=True, diag=True)
    return a, 0.6, np.random.default_rng(2).standard_normal(a.n)


def test_forward_strang_level0_is_the_dense_column_split():
    # Level 0 (one step, dt = t): e^{t D'/2} e^{t M} e^{t D'/2} v with
    # D'_i = a_ii + sum_{k != i} |a_ki| (column sums of |A|) and M the
    # off-diagonal part of A minus diag of those column sums.
    a, t, v = _nonsym()
    dense = a.dense()
    off = dense - np.diag(np.diag(dense))
    colsum = np.abs(off).sum(axis=0)
    m = off - np.diag(colsum)
    e = np.exp(t * (np.diag(dense) + colsum) / 2.0)
    want = e * (R.expm_pade13(t * m) @ (e * v))
    got = R.strang_forward(a.scipy(), t, v, 0)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_forward_strang_converges_at_second_order():
    a, t, v = _nonsym()
    ref = R.expmv(a.scipy(), t, v)
    errs = [np.linalg.norm(R.strang_forward(a.scipy(), t, v, l) - ref) for l in range(3, 8)]
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.2), ratios


def test_forward_and_backward_means_agree_for_symmetric_a():
    a = I.laplacian_2d(6)
    v = np.random.default_rng(1).random(a.n)
    for l in (0, 2):
        f = R.strang_forward(a.scipy(), 0.3, v, l)
        b = R.strang(a.scipy(), 0.3, v, l)
        assert np.abs(f - b).max() <= 1e-14 * np.abs(b).max()


def test_start_weights_are_exact_integers():
    v = np.array([2.0, -1.0, 0.0, 1e-30, 0.3, -2.0])
    w, cdf, total = W.start_weights(v)
    assert w.tolist() == [1 << 20, 1 << 19, 0, 1, int(np.ceil(0.15 * (1 << 20))), 1 << 20]
    assert cdf.tolist() == np.cumsum(w).tolist() and total == int(w.sum())


def test_start_law_and_zero_entries():
    a, t, _ = _nonsym()
    v = np.random.default_rng(4).standard_normal(a.n)
    v[::5] = 0.0
    fw = W.ForwardWalker(a, t, v, seed=11)
    m = 100000
    rec = fw.walks_fwd(0, m, 0, False)
    cnt = np.bincount(rec["pad"], minlength=a.n)
    p = fw.w / fw.W
    assert cnt[p == 0].sum() == 0
    pos = p > 0
    chi2 = (((cnt[pos] - m * p[pos]) ** 2) / (m * p[pos])).sum()
    dof = int((p > 0).sum()) - 1
    assert chi2 < dof + 6.0 * np.sqrt(2.0 * dof), chi2


def test_diagonal_matrix_forward_walks_are_exact():
    d = np.linspace(-1.0, 0.5, 16)
    a = I.to_csr(sp.diags(d).tocsr())
    v = np.random.default_rng(3).standard_normal(16)
    fw = W.ForwardWalker(a, 0.7, v, seed=5)
    rec = fw.walks_fwd(0, 2000, 2, False)
    s = rec["pad"]
    assert np.array_equal(rec["end"], s) and np.all(rec["jumps"] == 0)
    want = v[s] * (fw.W / fw.w[s]) * np.exp(0.7 * d[s])
    assert np.abs(rec["y"] - want).max() <= 1e-13 * np.abs(want).max()


def test_column_stochastic_generator_conserves_mass_per_walk():
    # A = -L (graph Laplacian): columns of A^T's split have d' = 0, so every
    # forward walk carries exactly v_s W / w_s and 1^T x-hat = 1^T v exactly in
    # expectation (1^T exp(tA) = 1^T).
    a = I.ba_graph(200, 3, seed=6)
    lap = -(sp.diags(np.diff(a.row_ptr).astype(float)) - a.scipy())
    a2 = I.to_csr(lap.tocsr())
    v = np.random.default_rng(7).standard_normal(a2.n)
    fw = W.ForwardWalker(a2, 0.5, v, seed=9)
    rec = fw.walks_fwd(0, 4000, 3, False)
    s = rec["pad"]
    want = v[s] * (fw.W / fw.w[s])
    assert np.abs(rec["y"] - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("level,coarse", [(0, False), (2, False), (2, True)])
def test_forward_level_means_match_strang(level, coarse):
    a, t, v = _nonsym()
    want = R.strang_forward(a.scipy(), t, v, level)
    if coarse:
        want = want - R.strang_forward(a.scipy(), t, v, level - 1)
    fw = W.ForwardWalker(a, t, v, seed=3 + level)
    m = 200000
    rec = fw.walks_fwd(0, m, level, coarse)
    z1 = np.zeros(a.n)
    z2 = np.zeros(a.n)
    np.add.at(z1, rec["end"], rec["y"])
    np.add.at(z2, rec["end"], rec["y"] ** 2)
    mean = z1 / m
    se = np.sqrt(np.maximum(z2 / m - mean ** 2, 0.0) / m)
    ok = se > 0
    z = (mean - want)[ok] / se[ok]
    assert np.abs(z).max() < 5.0 and np.sqrt((z ** 2).mean()) < 1.5, np.abs(z).max()
    assert np.all(np.abs(mean - want)[~ok] <= 1e-12 * np.abs(v).max())


def test_forward_importance_sampling_is_unbiased():
    a, t, v = _nonsym()
    level = 1
    want = R.strang_forward(a.scipy(), t, v, level)
    h = np.random.default_rng(12).uniform(0.2, 3.0, a.n)
    fw = W.ForwardWalker(a, t, v, seed=21, h=h, alpha=0.2)
    m = 200000
    rec = fw.walks_fwd(0, m, level, False)
    z1 = np.zeros(a.n)
    z2 = np.zeros(a.n)
    np.add.at(z1, rec["end"], rec["y"])
    np.add.at(z2, rec["end"], rec["y"] ** 2)
    mean = z1 / m
    se = np.sqrt(np.maximum(z2 / m - mean ** 2, 0.0) / m)
    z = (mean - want) / se
    assert np.abs(z).max() < 5.0, np.abs(z).max()


def test_forward_walks_are_counter_addressed():
    a, t, v = _nonsym()
    fw = W.ForwardWalker(a, t, v, seed=17)
    whole = fw.walks_fwd(0, 300, 2, True)
    part = fw.walks_fwd(123, 50, 2, True)
    assert np.array_equal(whole[123:173], part)
    sx, _, _, _ = fw.mlmcl_fwd(2, True, 0, 300)
    acc = np.zeros(a.n)
    np.add.at(acc, whole["end"], whole["y"])
    assert np.abs(sx - acc).max() <= 1e-12 * max(1.0, np.abs(acc).max())
