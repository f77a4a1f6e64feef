"""Pins for the oracle's MLP reference: its analytic gradient against
central finite differences of its own loss (rounding off), and the BF16
rounding helper against exact cases."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_is_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-3])
    got = mlp.round_bf16(vals)
    # BF16 keeps 7 fraction bits: the step at 1.0 is 2^-7
    assert got[0] == 1.0
    assert got[1] == 1.0               # exactly half a step: tie goes to the even value 1.0
    assert got[2] == 1.0               # below half a step
    assert got[3] == 1.0 + 2 ** -7     # above half a step
    assert got[4] == -2.5
    assert abs(got[5] - 3.0e-3) <= 2 ** -8 * 3.0e-3


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.N_PARAMS) * 0.3
    x = rng.standard_normal((37, mlp.N_IN))
    y = rng.standard_normal(37)
    _, _, g = mlp.loss_and_grad(p, x, y, bf16=False)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (mlp.loss_and_grad(pp, x, y, bf16=False)[1] - mlp.loss_and_grad(pm, x, y, bf16=False)[1]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * (1 + abs(num)), (i, num, g[i])
