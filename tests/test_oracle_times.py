"""Pins of the oracle's intermediate-time samples (Sec. 5, Fig. 7; Algorithm
3 evaluates the Strang weight at every grid time of a walk).

A walk's sample for t_k = t k/T is formed from its prefix up to the fine grid
point k N/T.  Its mean must be the level-l Strang product of k N/T steps of
dt = t/N (Eq. 2), computed here step by step by an independent route
(reference.strang_times); the coupled (fine minus coarse) prefix sample's
mean must be the difference of the two levels' products at that time; the
last time is the walk's own sample; and the prefix of a walk at level l up to
s = 1/2 has the law of a whole walk of the half-time problem at level l-1,
so their exact means agree (a closed-form identity of the split).
"""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W


def _problem():
    a = I.random_sparse(9, 3, seed=21, signed=True, diag=True)
    return a, 0.9, np.random.default_rng(4).random(9) - 0.3


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
@pytest.mark.parametrize("level,coarse,n_times", [(2, False, 4), (3, False, 2), (4, True, 8),
                                                 (3, True, 4)])
def test_prefix_means_are_the_strang_products_at_the_times(precision, level, coarse, n_times):
    a, t, v = _problem()
    reps = 1 << 16
    wk = W.Walker(a, t, v, seed=88, precision=precision)
    rows = np.repeat(np.arange(a.n), reps)
    rr = np.tile(np.arange(reps), a.n)
    rec, yt = wk.walks_times(rows, rr, level, coarse, n_times)
    want = R.strang_times(a.scipy(), t, v, level, n_times)
    if coarse:
        want = want - R.strang_times(a.scipy(), t, v, level - 1, n_times)
    for k in range(n_times - 1):
        y = yt[:, k].reshape(a.n, reps)
        m = y.mean(axis=1)
        se = y.std(axis=1) / np.sqrt(reps)
        ok = se > 1e-12 * np.abs(m)     # rows that never jump are deterministic
        z = (m[ok] - want[k][ok]) / se[ok]
        assert np.all(np.abs(z) < 4.5), (k, z)
        assert np.allclose(m[~ok], want[k][~ok], rtol=1e-9, atol=1e-12)
    # the last time is the walk's own sample (the product of all N steps)
    assert np.allclose(rec["y"].reshape(a.n, reps).mean(axis=1), want[-1],
                       atol=5 * rec["y"].reshape(a.n, reps).std(axis=1).max() / np.sqrt(reps))


def test_half_time_prefix_is_the_half_time_problem():
    # the prefix to s = 1/2 at level l with time t has the law of a whole
    # walk of time t/2 at level l - 1: the same exact mean
    a, t, v = _problem()
    for level in (1, 2, 4):
        half = R.strang_times(a.scipy(), t, v, level, 2)[0]
        whole = R.strang(a.scipy(), t / 2, v, level - 1)
        assert np.allclose(half, whole, rtol=1e-13, atol=1e-14)


def test_walk_limit_keeps_the_passed_times():
    # a walk stopped at the jump limit keeps the samples of the times before
    # the stop and has 0 at the later ones and at the end
    a = I.laplacian_2d(6, 1.0)
    t, v = 2.0, np.random.default_rng(2).random(a.n)
    wk = W.Walker(a, t, v, seed=3, max_jumps=3)
    rec, yt = wk.walks_times(np.arange(a.n), np.zeros(a.n, np.int64), 4, False, 8)
    lim = rec["status"] == 1
    assert lim.any()
    assert np.all(rec["y"][lim] == 0.0)
    assert np.any(yt[lim, 0] != 0.0)        # the first time is passed before 3 jumps
    full = W.Walker(a, t, v, seed=3)
    rec2, yt2 = full.walks_times(np.arange(a.n), np.zeros(a.n, np.int64), 4, False, 8)
    # the samples before the stop are those of the unlimited walk
    for i in np.flatnonzero(lim):
        nz = yt[i] != 0.0
        assert np.array_equal(yt[i][nz], yt2[i][nz])
