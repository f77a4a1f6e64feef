"""Deterministic FP64 references for x = exp(t A) v and its MLMC levels.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Everything here is the plain definition written out with dense or sparse
matrix products as the only library primitives:

* :func:`split` -- the splitting A = D - T of Sec. 2.1 (Eq. 1).
* :func:`expm_pade13` -- exp(M) by scaling and squaring with the diagonal
  [13/13] Pade approximant (Higham, SIAM J. Matrix Anal. Appl. 26 (2005)),
  for the dense n <= 4096 judge.
* :func:`expmv_taylor` -- exp(tA)v by truncated Taylor series with s
  substeps, s = ceil(t ||A||_1) (the scaling idea of Al-Mohy and Higham 2011,
  cited by the paper), terms added until the last one is below 2^-53 of the
  partial sum in the max norm.
* :func:`strang` -- the level-l approximation of Eq. 2,
  (e^{dt D/2} e^{-dt T} e^{dt D/2})^N v with N = 2^l and dt = t/N.
* :func:`level_moments` -- exact E[Y] and E[Y^2] per start row for the
  level-l correction Y of Algorithm 2, by transfer matrices over the grid
  points (the walk's skeleton is a Markov chain with kernel exp(dt Q)).
* :func:`brute_moments` -- the same by enumerating every skeleton path
  (tiny n and N only).
* :func:`dst_expmv_laplacian_2d` -- the closed form of exp(tA)v for the 2D
  Dirichlet Laplacian by its sine eigenbasis.
* :func:`strang_source`, :func:`expmv_source_exact` -- the level-l mean of
  Algorithm 3's Simpson source term and the exact int_0^t exp(sA) f ds.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla


# ---------------------------------------------------------------------------
# Splitting (Sec. 2.1, Eq. 1)
# ---------------------------------------------------------------------------
def split(a_dense: np.ndarray):
    """Return (d, Lii, T, sigma) with d_i = a_ii + L_ii, L_ii = sum_{j!=i}
    |a_ij|, sigma_ij = [a_ij < 0], and T_ii = L_ii, T_ij = (-1)^sigma_ij L_ij
    where L_ij = -|a_ij|, so that A = diag(d) - T."""
    a = np.asarray(a_dense, dtype=np.float64)
    n = a.shape[0]
    off = a.copy()
    np.fill_diagonal(off, 0.0)
    lap_off = -np.abs(off)                       # L_ij, i != j
    lii = -lap_off.sum(axis=1)                   # zero row sums
    sigma = (off < 0).astype(np.int64)
    t = np.where(sigma == 1, -1.0, 1.0) * lap_off
    t[np.arange(n), np.arange(n)] = lii
    d = np.diag(a) + lii
    return d, lii, t, sigma


def generators(a_dense: np.ndarray, t: float):
    """Scaled-time generators of the walk: Q = -t L (unsigned, rows sum to
    zero) and Qs = -t T (signed: off-diagonals t a_ij, diagonal -t L_ii),
    and the scaled diagonal dl = t d."""
    d, lii, tmat, _ = split(a_dense)
    n = a_dense.shape[0]
    off = np.abs(np.asarray(a_dense, dtype=np.float64))
    np.fill_diagonal(off, 0.0)
    q = t * off
    q[np.arange(n), np.arange(n)] = -t * lii
    return q, -t * tmat, t * d


# ---------------------------------------------------------------------------
# exp(M): Pade-13 scaling and squaring
# ---------------------------------------------------------------------------
_PADE_M = 13
# b_j = (2m-j)! m! / ((2m)! j! (m-j)!), the numerator of the [m/m] Pade
# approximant of e^x (the denominator is the same polynomial at -x).
_PADE_B = [float(Fraction(math.factorial(2 * _PADE_M - j) * math.factorial(_PADE_M),
                          math.factorial(2 * _PADE_M) * math.factorial(j)
                          * math.factorial(_PADE_M - j))) for j in range(_PADE_M + 1)]
_THETA_13 = 5.371920351148152


def expm_pade13(m: np.ndarray) -> np.ndarray:
    """exp(M) for a dense square matrix: scale by 2^-s so that ||M/2^s||_1 <=
    theta_13, evaluate r_13 = q(-M)^{-1} q(M) with q(x) = sum b_j x^j, then
    square s times."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    norm1 = np.abs(m).sum(axis=0).max() if n else 0.0
    s = 0 if norm1 <= _THETA_13 else int(math.ceil(math.log2(norm1 / _THETA_13)))
    a = m / (2.0 ** s)
    b = _PADE_B
    ident = np.eye(n)
    a2 = a @ a
    a4 = a2 @ a2
    a6 = a4 @ a2
    u = a @ (a6 @ (b[13] * a6 + b[11] * a4 + b[9] * a2)
             + b[7] * a6 + b[5] * a4 + b[3] * a2 + b[1] * ident)
    v = a6 @ (b[12] * a6 + b[10] * a4 + b[8] * a2) + b[6] * a6 + b[4] * a4 + b[2] * a2 \
        + b[0] * ident
    r = np.linalg.solve(v - u, v + u)
    for _ in range(s):
        r = r @ r
    return r


# ---------------------------------------------------------------------------
# exp(tA) v: truncated Taylor with substeps
# ---------------------------------------------------------------------------
def expmv_taylor(a, t: float, v: np.ndarray, max_terms: int = 200) -> np.ndarray:
    """exp(tA)v for a sparse or dense A: s = max(1, ceil(t ||A||_1))
    substeps of length h = t/s; in each, w <- sum_k (hA)^k w / k! until two
    consecutive terms are <= 2^-53 ||partial sum||_inf."""
    if sp.issparse(a):
        a = sp.csr_matrix(a, dtype=np.float64)
        norm1 = float(abs(a).sum(axis=0).max()) if a.shape[0] else 0.0
    else:
        a = np.asarray(a, dtype=np.float64)
        norm1 = float(np.abs(a).sum(axis=0).max()) if a.shape[0] else 0.0
    w = np.array(v, dtype=np.float64, copy=True)
    if t == 0.0 or norm1 == 0.0:
        return w
    s = max(1, int(math.ceil(abs(t) * norm1)))
    h = t / s
    for _ in range(s):
        acc = w.copy()
        term = w
        small = 0
        for k in range(1, max_terms + 1):
            term = (h * (a @ term)) / k
            acc = acc + term
            if np.abs(term).max() <= 2.0 ** -53 * np.abs(acc).max():
                small += 1
                if small == 2:
                    break
            else:
                small = 0
        w = acc
    return w


def expmv(a, t: float, v: np.ndarray) -> np.ndarray:
    """FP64 judge of exp(tA)v: dense Pade-13 for n <= 4096, Taylor above."""
    n = a.shape[0]
    if n <= 4096:
        dense = a.toarray() if sp.issparse(a) else np.asarray(a, dtype=np.float64)
        return expm_pade13(t * dense) @ np.asarray(v, dtype=np.float64)
    return expmv_taylor(a, t, v)


# ---------------------------------------------------------------------------
# Strang levels (Eq. 2) and the telescoping corrections (Eq. 8-9)
# ---------------------------------------------------------------------------
def _split_sparse(a, lam=None):
    """Sparse splitting: returns (d, -T as sparse) of Eq. 1.  With ``lam``
    (the rates of a walk with tilted clocks) the split A = D' - T' with
    D' = diag(a_ii + lam_i) and -T' = (A - diag(a)) - diag(lam)."""
    a = sp.csr_matrix(a, dtype=np.float64)
    diag = a.diagonal()
    off = a - sp.diags(diag)
    off.eliminate_zeros()
    lii = np.asarray(abs(off).sum(axis=1)).ravel() if lam is None else np.asarray(lam, float)
    minus_t = (off - sp.diags(lii)).tocsr()      # off-diagonals a_ij, diagonal -L_ii
    return diag + lii, minus_t


def strang(a, t: float, v: np.ndarray, level: int, lam=None) -> np.ndarray:
    """x-bar of Eq. 2 with N = 2^level steps of dt = t/N:
    apply e^{dt D/2} e^{-dt T} e^{dt D/2} N times to v.  With ``lam``: the
    same product for the split of a walk with rates lam (_split_sparse),
    which is what a walk with tilted clocks estimates at level l."""
    n_steps = 1 << level
    dt = t / n_steps
    d, minus_t = _split_sparse(a, lam)
    half = np.exp(dt * d / 2.0)
    dense = None
    if a.shape[0] <= 2048:
        dense = expm_pade13(dt * minus_t.toarray())
    w = np.array(v, dtype=np.float64, copy=True)
    for _ in range(n_steps):
        w = half * w
        w = dense @ w if dense is not None else expmv_taylor(minus_t, dt, w)
        w = half * w
    return w


def strang_times(a, t: float, v: np.ndarray, level: int, n_times: int, lam=None) -> np.ndarray:
    """The level-l Strang product at the times t k / n_times, k = 1..n_times:
    row k-1 holds (e^{dt D/2} e^{-dt T} e^{dt D/2})^{k N / n_times} v with
    N = 2^level, dt = t/N (the mean of a walk's prefix sample at that time)."""
    n_steps = 1 << level
    if n_steps % n_times:
        raise ValueError("n_times must divide 2^level")
    dt = t / n_steps
    d, minus_t = _split_sparse(a, lam)
    half = np.exp(dt * d / 2.0)
    dense = expm_pade13(dt * minus_t.toarray()) if a.shape[0] <= 2048 else None
    w = np.array(v, dtype=np.float64, copy=True)
    out = []
    stride = n_steps // n_times
    for step in range(1, n_steps + 1):
        w = half * w
        w = dense @ w if dense is not None else expmv_taylor(minus_t, dt, w)
        w = half * w
        if step % stride == 0:
            out.append(w.copy())
    return np.array(out)


def strang_forward(a, t: float, v: np.ndarray, level: int) -> np.ndarray:
    """Mean of the forward-mode level-l estimate (Eq. 5 read on B = A^T):
    with B = D' - T' split by Eq. 1 (d'_i = a_ii + sum_{k != i} |a_ki|), the
    backward Strang operator of B is S_B = (e^{dt D'/2} e^{-dt T'} e^{dt D'/2})^N
    and the forward walks estimate S_B^T v; S_B^T applies e^{-dt T'^T}, whose
    off-diagonals are a_ij and diagonal -L'_ii."""
    n_steps = 1 << level
    dt = t / n_steps
    b = sp.csr_matrix(a, dtype=np.float64).T.tocsr()
    d_b, minus_tb = _split_sparse(b)          # d' and -T' (of B)
    minus_tbt = minus_tb.T.tocsr()            # -T'^T
    half = np.exp(dt * d_b / 2.0)
    dense = expm_pade13(dt * minus_tbt.toarray()) if a.shape[0] <= 2048 else None
    w = np.array(v, dtype=np.float64, copy=True)
    for _ in range(n_steps):
        w = half * w
        w = dense @ w if dense is not None else expmv_taylor(minus_tbt, dt, w)
        w = half * w
    return w


def _strang_step_operator(a, dt: float):
    """One step of Eq. 2 as a callable w -> e^{dt D/2} e^{-dt T} e^{dt D/2} w."""
    d, minus_t = _split_sparse(a)
    half = np.exp(dt * d / 2.0)
    dense = expm_pade13(dt * minus_t.toarray()) if a.shape[0] <= 2048 else None

    def step(w):
        w = half * w
        w = dense @ w if dense is not None else expmv_taylor(minus_t, dt, w)
        return half * w
    return step


def strang_source(a, t: float, f: np.ndarray, level: int, coarse: bool = False) -> np.ndarray:
    """Mean of the source part of Algorithm 3 at level l (reading R17): the
    Simpson rule (h/3) sum_{n=0}^{K} w_n S^n f over K steps of length h with
    weights 1, 4, 2, 4, ..., 4, 1, where S is the one-step Strang operator of
    Eq. 2 for step h.  coarse=False: K = N = 2^level, h = t/N; coarse=True:
    the same path's level-(l-1) rule, K = N/2, h = 2t/N.  K must be even."""
    n_steps = (1 << level) // (2 if coarse else 1)
    if n_steps < 2 or n_steps % 2:
        raise ValueError("Simpson's rule needs an even number of steps >= 2")
    h = t / n_steps
    step = _strang_step_operator(sp.csr_matrix(a, dtype=np.float64), h)
    w = np.array(f, dtype=np.float64, copy=True)
    acc = w.copy()                              # n = 0, weight 1
    for k in range(1, n_steps + 1):
        w = step(w)
        weight = 1.0 if k == n_steps else (4.0 if k % 2 else 2.0)
        acc = acc + weight * w
    return (h / 3.0) * acc


def expmv_source_exact(a, t: float, f: np.ndarray) -> np.ndarray:
    """int_0^t exp(sA) f ds, from the exponential of the augmented matrix
    [[tA, t f], [0, 0]] (its top-right column; dense, n <= 4096)."""
    dense = a.toarray() if sp.issparse(a) else np.asarray(a, dtype=np.float64)
    n = dense.shape[0]
    m = np.zeros((n + 1, n + 1))
    m[:n, :n] = t * dense
    m[:n, n] = t * np.asarray(f, dtype=np.float64)
    return expm_pade13(m)[:n, n]


def expmv_source_taylor(a, t: float, f: np.ndarray) -> np.ndarray:
    """int_0^t exp(sA) f ds for large sparse A: exp(t B) applied to e_{n+1}
    with the sparse augmented B = [[A, f], [0, 0]] (truncated Taylor with
    substeps), top n entries."""
    a = sp.csr_matrix(a, dtype=np.float64)
    n = a.shape[0]
    col = sp.csr_matrix(np.asarray(f, dtype=np.float64).reshape(n, 1))
    b = sp.bmat([[a, col], [None, sp.csr_matrix((1, 1))]], format="csr")
    e = np.zeros(n + 1)
    e[n] = 1.0
    return expmv_taylor(b, t, e)[:n]


def level_means(a, t: float, v: np.ndarray, l0: int, top: int, lam=None):
    """Exact per-level corrections m_l of Eq. 9 for l = l0..top:
    m_l0 = x-bar^(l0), m_l = x-bar^(l) - x-bar^(l-1) (``lam``: the split of
    a walk with tilted clocks)."""
    xs = {l: strang(a, t, v, l, lam) for l in range(max(0, l0 - 1) if l0 > 0 else 0, top + 1)}
    out = {l0: xs[l0]}
    for l in range(l0 + 1, top + 1):
        out[l] = xs[l] - xs[l - 1]
    return out


# ---------------------------------------------------------------------------
# Exact moments of one level's correction (Lemma 1-2)
# ---------------------------------------------------------------------------
def _weights(level: int, coarse: bool):
    """Exponent weights c_k on grid points k = 0..N (scaled time, dl units):
    fine c_f = (1/2, 1, ..., 1, 1/2)/N; coarse (level - 1 on even points)
    c_c = (1, 0, 2, 0, ..., 2, 0, 1)/N."""
    n = 1 << level
    cf = np.full(n + 1, 1.0 / n)
    cf[0] = cf[-1] = 0.5 / n
    if not coarse:
        return cf, None
    cc = np.zeros(n + 1)
    cc[0::2] = 2.0 / n
    cc[0] = cc[-1] = 1.0 / n
    return cf, cc


def _functional(kernel: np.ndarray, dl: np.ndarray, c: np.ndarray, g: np.ndarray):
    """F_i = E_i[exp(sum_k c_k dl_{X_k}) g(X_N)] for the chain with one-step
    kernel ``kernel``: D_0 K D_1 K ... K D_N g."""
    w = np.exp(c[-1] * dl) * g
    for k in range(len(c) - 2, -1, -1):
        w = np.exp(c[k] * dl) * (kernel @ w)
    return w


def tilt_law(a_dense: np.ndarray, h: np.ndarray, alpha: float, t: float):
    """The h-transform walk's law in FP64 (no table rounding): rates
    lam_i = sum_{j != i} |a_ij| h_j / h_i clamped to [L_ii/1024,
    max(L_ii, 2/t)] (0 where L_ii = 0) and jump law q_ij = (1 - alpha)
    |a_ij| h_j / sum_k |a_ik| h_k + alpha |a_ij| / L_ii (rows with L_ii = 0:
    zero)."""
    a = np.asarray(a_dense, dtype=np.float64)
    off = np.abs(a.copy())
    np.fill_diagonal(off, 0.0)
    h = np.asarray(h, dtype=np.float64)
    lii = off.sum(axis=1)
    hs = off @ h
    q = np.zeros_like(off)
    lam = np.zeros(a.shape[0])
    rows = lii > 0
    q[rows] = ((1.0 - alpha) * off[rows] * h[None, :] / hs[rows, None]
               + alpha * off[rows] / lii[rows, None])
    cap = 2.0 / t if t > 0 else 0.0
    lam[rows] = np.clip(hs[rows] / h[rows], lii[rows] / 1024.0, np.maximum(lii[rows], cap))
    return lam, q


def walk_generators(a_dense: np.ndarray, t: float, lam=None, q=None):
    """Scaled-time generators of a walk with rates lam and jump law q that
    carries the factor a_jk / (lam_j q_jk) per jump (lam = L, q = k: the
    paper's walk, generators()): the mean's kernel generator t (N - diag lam)
    with N the off-diagonal part of A (signed), the second moment's
    t (R2 - diag lam) with R2_jk = a_jk^2 / (lam_j q_jk) (the squared factor
    times the jump rate), and dl = t (a_ii + lam_i)."""
    a = np.asarray(a_dense, dtype=np.float64)
    n = a.shape[0]
    off = a.copy()
    np.fill_diagonal(off, 0.0)
    if lam is None:
        lam = np.abs(off).sum(axis=1)
    if q is None:
        with np.errstate(divide="ignore", invalid="ignore"):
            q = np.where(lam[:, None] > 0, np.abs(off) / lam[:, None], 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        r2 = np.where((off != 0) & (q > 0), off * off / (lam[:, None] * q), 0.0)
    g1 = t * (off - np.diag(lam))
    g2 = t * (r2 - np.diag(lam))
    return g1, g2, t * (np.diag(a) + lam)


def level_moments(a_dense: np.ndarray, t: float, v: np.ndarray, level: int, coarse: bool,
                  lam=None, q=None):
    """Exact (E[Y], E[Y^2]) per start row for the level-``level`` sample of
    Algorithm 2: Y = phi v_{X_N} (e^{E_f} - e^{E_c}) when ``coarse``, else
    phi v_{X_N} e^{E_f}.  The mean uses the signed kernel exp(dt Qs); the
    second moment uses the unsigned exp(dt Q), since phi^2 = 1 and fine and
    coarse share phi.  With ``lam`` and ``q`` the walk has tilted clocks and
    jumps (walk_generators): the kernels are exp(dt G1) and exp(dt G2)."""
    if lam is not None or q is not None:
        g1, g2, dl = walk_generators(a_dense, t, lam, q)
        n_steps = 1 << level
        ks = expm_pade13(g1 / n_steps)
        ku = expm_pade13(g2 / n_steps)
        return _moments_from_kernels(ks, ku, dl, v, level, coarse)
    q, qs, dl = generators(a_dense, t)
    n_steps = 1 << level
    ks = expm_pade13(qs / n_steps)
    ku = expm_pade13(q / n_steps)
    return _moments_from_kernels(ks, ku, dl, v, level, coarse)


def _moments_from_kernels(ks, ku, dl, v, level: int, coarse: bool):
    """(E[Y], E[Y^2]) from the one-step kernels of the mean and of the
    second moment over the N = 2^level grid steps."""
    v = np.asarray(v, dtype=np.float64)
    cf, cc = _weights(level, coarse)
    if not coarse:
        m1 = _functional(ks, dl, cf, v)
        m2 = _functional(ku, dl, 2 * cf, v * v)
        return m1, m2
    m1 = _functional(ks, dl, cf, v) - _functional(ks, dl, cc, v)
    m2 = (_functional(ku, dl, 2 * cf, v * v) - 2.0 * _functional(ku, dl, cf + cc, v * v)
          + _functional(ku, dl, 2 * cc, v * v))
    return m1, m2


def _functional_pieces(kernels, dls, c: np.ndarray, g: np.ndarray, per: int):
    """_functional with a law per time piece (reading R19): the step over
    interval k+1 (from grid point k to k+1) uses the kernel of its piece
    k // per; grid point k takes half of its weight c_k from each adjacent
    interval's piece (all of it at the ends 0 and N), so a point on a piece
    boundary gets the mean of the two pieces' dl."""
    n_steps = c.size - 1
    piece = lambda interval: (interval - 1) // per  # interval = 1..N
    w = np.exp(c[n_steps] * dls[piece(n_steps)]) * g
    for k in range(n_steps - 1, -1, -1):
        right = piece(k + 1)
        w = kernels[right] @ w
        if k == 0:
            e = c[0] * dls[right]
        else:
            e = 0.5 * c[k] * (dls[piece(k)] + dls[right])
        w = np.exp(e) * w
    return w


def level_moments_pieces(a_dense: np.ndarray, t: float, v: np.ndarray, level: int,
                         coarse: bool, laws):
    """level_moments for a walk whose law changes with time (reading R19):
    ``laws`` holds K pairs (lam, q), pair p for the scaled times
    [p/K, (p+1)/K); N = 2^level must be a multiple of K."""
    n_steps = 1 << level
    k_pieces = len(laws)
    if n_steps % k_pieces:
        raise ValueError("the grid must hold every piece boundary")
    ks, ku, dls = [], [], []
    for lam, q in laws:
        g1, g2, dl = walk_generators(a_dense, t, lam, q)
        ks.append(expm_pade13(g1 / n_steps))
        ku.append(expm_pade13(g2 / n_steps))
        dls.append(dl)
    per = n_steps // k_pieces
    v = np.asarray(v, dtype=np.float64)
    cf, cc = _weights(level, coarse)
    f = lambda kern, c, g: _functional_pieces(kern, dls, c, g, per)
    if not coarse:
        return f(ks, cf, v), f(ku, 2 * cf, v * v)
    m1 = f(ks, cf, v) - f(ks, cc, v)
    m2 = f(ku, 2 * cf, v * v) - 2.0 * f(ku, cf + cc, v * v) + f(ku, 2 * cc, v * v)
    return m1, m2


def brute_moments(a_dense: np.ndarray, t: float, v: np.ndarray, level: int, coarse: bool):
    """(E[Y], E[Y^2]) per start row by summing over every skeleton path
    (X_1, ..., X_N) in {0..n-1}^N with probability prod K(X_{k-1}, X_k)
    (signed kernel for the mean, unsigned for the second moment)."""
    q, qs, dl = generators(a_dense, t)
    n = a_dense.shape[0]
    n_steps = 1 << level
    ks = expm_pade13(qs / n_steps)
    ku = expm_pade13(q / n_steps)
    cf, cc = _weights(level, coarse)
    m1 = np.zeros(n)
    m2 = np.zeros(n)
    for i in range(n):
        for path in itertools.product(range(n), repeat=n_steps):
            states = (i,) + path
            ps = 1.0
            pu = 1.0
            for k in range(n_steps):
                ps *= ks[states[k], states[k + 1]]
                pu *= ku[states[k], states[k + 1]]
            ef = sum(cf[k] * dl[s] for k, s in enumerate(states))
            vend = v[states[-1]]
            if coarse:
                ec = sum(cc[k] * dl[s] for k, s in enumerate(states))
                y = vend * (math.exp(ef) - math.exp(ec))
            else:
                y = vend * math.exp(ef)
            m1[i] += ps * y
            m2[i] += pu * y * y
    return m1, m2


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------
def dst_expmv_laplacian_2d(g: int, scale: float, t: float, v: np.ndarray) -> np.ndarray:
    """exp(t * scale * L5) v for the g x g Dirichlet 5-point Laplacian L5
    (row index ix*g + iy) from its eigenbasis: S_kp = sqrt(2/(g+1))
    sin(k p pi/(g+1)), eigenvalues -4 + 2cos(p pi/(g+1)) + 2cos(q pi/(g+1))."""
    k = np.arange(1, g + 1)
    s = np.sqrt(2.0 / (g + 1)) * np.sin(np.outer(k, k) * np.pi / (g + 1))
    lam1 = -2.0 + 2.0 * np.cos(k * np.pi / (g + 1))
    lam = lam1[:, None] + lam1[None, :]
    vm = np.asarray(v, dtype=np.float64).reshape(g, g)
    coef = s @ vm @ s
    return (s @ (np.exp(t * scale * lam) * coef) @ s).ravel()


def level_variance_total(m1: np.ndarray, m2: np.ndarray) -> float:
    """V_l as the scalar total variance sum_i (E[Y_i^2] - E[Y_i]^2)."""
    return float(np.sum(m2 - m1 * m1))


def choose_l0(d: np.ndarray, lii: np.ndarray, t: float) -> int:
    """Coarsest level by Eq. 16, l0 = log2(2 beta d_max), read with d_max =
    max_i max(|d_i|, L_ii) and rounded up, never below 0."""
    dm = float(np.max(np.maximum(np.abs(d), lii))) if d.size else 0.0
    if dm * t <= 0.0:
        return 0
    return max(0, int(math.ceil(math.log2(2.0 * t * dm))))
