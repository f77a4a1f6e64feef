"""Pins for the oracle's random-number pieces: Philox4x32-10, the uniforms
and neglog.  None of these compare the oracle with itself."""
import os

import numpy as np
import pytest

from oracle import walker as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [int(x, 16) for x in line.split()]
        rows.append((f[0:4], f[4:6], f[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(W.philox(ctr, key)) == out


def test_philox_uniformity_and_counter_sensitivity():
    # 2^14 counters: every output word is uniform (chi-square over 16 bins)
    # and flipping one counter bit changes about half of the 128 output bits.
    outs = np.array([W.philox([k, 7, 0, 1], [123, 456]) for k in range(1 << 14)],
                    dtype=np.uint64)
    for w in range(4):
        hist = np.bincount((outs[:, w] >> 28).astype(np.int64), minlength=16)
        e = outs.shape[0] / 16
        chi2 = float(((hist - e) ** 2 / e).sum())
        assert chi2 < 45.0  # 15 dof, p ~ 1e-4
    flips = []
    for k in range(256):
        a = W.philox([k, 1, 2, 3], [9, 9])
        b = W.philox([k ^ 0x10, 1, 2, 3], [9, 9])
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68


def test_uniforms_are_open_interval_and_exact():
    lib = W.lib()
    assert lib.orc_uniform64(0, 0) == 2.0 ** -53
    assert lib.orc_uniform64(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert lib.orc_uniform32(0) == np.float32(2.0 ** -24)
    assert lib.orc_uniform32(0xFFFFFFFF) == np.float32(1.0 - 2.0 ** -24)
    # odd multiples of 2^-53: the low bit of the mantissa numerator is set
    u = lib.orc_uniform64(0x12345678, 0x9ABCDEF0)
    k = u * 2.0 ** 53
    assert k == int(k) and int(k) % 2 == 1


def test_neglog64_accuracy():
    rng = np.random.default_rng(1)
    u = np.concatenate([rng.random(200_000), 2.0 ** -np.arange(1, 54),
                        1.0 - 2.0 ** -np.arange(1, 54),
                        [np.sqrt(0.5), np.nextafter(np.sqrt(0.5), 0), 0.5]])
    ref = -np.log(u)
    got = W.neglog64(u)
    assert np.all(got > 0)
    ulp = np.abs(got - ref) / np.spacing(ref)
    assert ulp.max() <= 4.0


def test_neglog32_accuracy():
    rng = np.random.default_rng(2)
    u = np.concatenate([rng.random(200_000).astype(np.float32),
                        (2.0 ** -np.arange(1, 25)).astype(np.float32),
                        (1.0 - 2.0 ** -np.arange(1, 25)).astype(np.float32),
                        np.array([np.sqrt(0.5), np.nextafter(np.float32(np.sqrt(0.5)), 0)],
                                 np.float32)])
    u = u[(u > 0) & (u < 1)]
    ref = -np.log(u.astype(np.float64))
    got = W.neglog32(u).astype(np.float64)
    assert np.all(got > 0)
    ulp = np.abs(got - ref) / np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert ulp.max() <= 1.0


def test_neglog32_within_one_ulp_on_every_fp32_uniform():
    # The walk's FP32 -ln(u) against the FP64 logarithm on all 2^23 uniforms
    # u = (2i+1) 2^-24 it is ever called with.
    i = np.arange(1 << 23, dtype=np.float64)
    u = ((2.0 * i + 1.0) * 2.0 ** -24).astype(np.float32)
    ref = -np.log(u.astype(np.float64))
    got = W.neglog32(u).astype(np.float64)
    ulp = np.abs(got - ref) / np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert ulp.max() <= 1.0


def test_exponential_law_of_holding_draws():
    # -ln(u) of the uniforms is Exp(1): mean 1, variance 1, and
    # P(E > 3) = e^-3 (Kolmogorov-Smirnov on 2^15 draws).
    lib = W.lib()
    xs = [W.philox([k, 0, 0, 0], [5, 6]) for k in range(1 << 15)]
    e = np.array([W.lib().orc_neglog64(lib.orc_uniform64(int(x[0]), int(x[1]))) for x in xs])
    e.sort()
    cdf = 1.0 - np.exp(-e)
    ks = np.max(np.abs(cdf - (np.arange(1, e.size + 1) / e.size)))
    assert ks < 1.63 / np.sqrt(e.size)  # alpha = 0.01


def test_neglog32_is_strictly_decreasing_over_every_fp32_uniform():
    # All 2^23 FP32 uniforms u = (2i+1) 2^-24: -ln(u) must decrease with i.
    # The GPU walk relies on it to decide "the first holding time reaches
    # s = 1" by comparing i with a per-row threshold index.
    i = np.arange(1 << 23, dtype=np.float64)
    u = ((2.0 * i + 1.0) * 2.0 ** -24).astype(np.float32)
    assert np.all(u.astype(np.float64) == (2.0 * i + 1.0) * 2.0 ** -24)
    g = W.neglog32(u).astype(np.float64)
    assert np.all(np.diff(g) < 0)


def _c_floats(path, start_marker, count):
    # The first `count` C hex-float literals after `start_marker` in a source
    # file, as FP32 values.
    import re
    text = open(path).read()
    body = text[text.index(start_marker):]
    lits = re.findall(r"-?0x1\.[0-9a-f]+p[-+]?\d+f", body)[:count]
    return np.array([float.fromhex(s[:-1]) for s in lits], np.float32)


def test_neglog32_coefficients_are_the_committed_fit():
    # R4: Q's FP32 coefficients are the relative-error least-squares fit on
    # Chebyshev points, rounded to FP32.  Re-running the fit must give exactly
    # the literals both sides compile (the oracle's C source and the walk
    # kernel's device header, each written on its own side).
    import os
    from oracle import fit_neglog32 as F
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    fitted = F.coefficients_fp32()
    orc = _c_floats(os.path.join(root, "oracle", "mlmc_oracle.c"), "orc_q32[ORC_NEGLOG_DEG32 + 1]", 9)
    dev = _c_floats(os.path.join(root, "paper_1904_12754_gb300", "csrc", "mlmc_device.cuh"),
                    "c[kNeglogDeg32 + 1]", 9)
    assert np.array_equal(fitted, orc)
    assert np.array_equal(fitted, dev)
    # the fit is insensitive to the number of nodes once it exceeds the degree
    assert np.array_equal(F.coefficients_fp32(64), fitted)
    # and every coefficient is well away from an FP32 rounding boundary, so a
    # different LAPACK cannot round it the other way
    c = F.fit()
    r = c.astype(np.float32).astype(np.float64)
    gap = np.abs(c - r) / np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
    assert np.all(gap < 0.45)
    # the printed literals parse back to the same values
    assert [float.fromhex(s[:-1]) for s in F.c_hex(fitted)] == [float(x) for x in fitted]
