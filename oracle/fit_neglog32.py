"""Fit of the FP32 -ln(u) polynomial (test infrastructure: the oracle's and
the walk kernel's FP32 -ln u both use these coefficients).

The paper draws exponential holding times (Sec. 3) without naming how -ln u
is computed; the reading used by both sides (R4) reduces u = m 2^e with
m in [sqrt(1/2), sqrt(2)), writes f = m - 1 and

    ln(1 + f) = f + f^2 Q(f),   Q of degree 8,

evaluated in FP32 by Horner's rule with fused multiply-adds.  Q's
coefficients are the least-squares fit, in FP64, of the RELATIVE error of
f + f^2 Q(f) against ln(1 + f) on the Chebyshev (Gauss) points
f_k = c + r cos((2k+1) pi / (2K)), k = 0..K-1 (K = 1000, c and r the centre
and half width of [sqrt(1/2) - 1, sqrt(2) - 1]), each rounded to the nearest
FP32 value.  Minimising

    sum_k ((f_k + f_k^2 Q(f_k) - ln(1 + f_k)) / ln(1 + f_k))^2

is linear in Q's coefficients: columns f_k^(2+i) / ln(1 + f_k), right-hand
side (ln(1 + f_k) - f_k) / ln(1 + f_k).  The solution is stable in K (any
K >= 16 gives the same FP32 values) and every coefficient lies at least
0.06 FP32 ulp away from a rounding boundary.

Run ``python -m oracle.fit_neglog32`` to print the coefficients as C hex
floats (constant term first).
"""
from __future__ import annotations

import numpy as np

DEGREE = 8
NODES = 1000


def fit(nodes: int = NODES, degree: int = DEGREE) -> np.ndarray:
    """FP64 least-squares coefficients of Q (constant term first)."""
    lo = float(np.sqrt(0.5)) - 1.0
    hi = float(np.sqrt(2.0)) - 1.0
    k = np.arange(nodes, dtype=np.float64)
    f = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos((2.0 * k + 1.0) * np.pi / (2.0 * nodes))
    f = f[f != 0.0]
    ln1p = np.log1p(f)
    cols = np.stack([f ** (2 + i) for i in range(degree + 1)], axis=1) / ln1p[:, None]
    rhs = (ln1p - f) / ln1p
    coef, *_ = np.linalg.lstsq(cols, rhs, rcond=None)
    return coef


def coefficients_fp32(nodes: int = NODES) -> np.ndarray:
    """Q's coefficients rounded to FP32 (the values the walks use)."""
    return fit(nodes).astype(np.float32)


def c_hex(values: np.ndarray) -> list[str]:
    """C99 hex-float literals with FP32 suffix, e.g. -0x1.fffff8p-2f."""
    out = []
    for v in values.astype(np.float64):
        m, e = np.frexp(abs(v))           # v = m 2^e, m in [0.5, 1)
        mant = int(round(m * 2.0 ** 24))  # 24 significant bits of an FP32 value
        frac = (mant - (1 << 23)) << 1    # 23 fraction bits as 6 hex digits
        s = f"{'-' if v < 0 else ''}0x1.{frac:06x}p{e - 1}f"
        out.append(s)
    return out


if __name__ == "__main__":
    print(", ".join(c_hex(coefficients_fp32())))
