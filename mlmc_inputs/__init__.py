"""Seeded synthetic inputs for the MLMC exp(tA)v estimator.

This module only builds matrices, times and right-hand sides: it holds none
of the estimator's arithmetic (no splitting, no transition law, no weights).
Both the CPU oracle's tests and the GPU path's tests and benchmark draw their
inputs from here, so the two sides see identical problems.

Every matrix is returned as canonical CSR (``row_ptr`` int64, ``col`` int32,
``val`` float64, columns strictly increasing within each row), which is the
layout the C-ABI library accepts.

Workload shapes follow the paper's benchmarks:
  * method-of-lines heat equation on a grid (Sec. 5, Example A, Eq. 19):
    5-point (2D) and 7-point (3D) Dirichlet Laplacians;
  * total communicability of a scale-free network (Sec. 5, Eq. 24): the
    paper's CONTEST ``pref`` networks are not available, so a seeded
    Barabasi-Albert graph stands in for them;
  * convection-diffusion (Sec. 5, Eq. 20-23): the paper's COMSOL FEM mesh is
    not available, so a 7-point upwind finite-difference operator on the
    paper's domain [-delta, delta]^3 stands in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

__all__ = [
    "CSR", "to_csr", "laplacian_2d", "laplacian_3d", "convdiff_3d", "ba_graph",
    "random_sparse", "star_graph", "ring_graph", "lambda_max", "uniform_v",
    "Workload", "workload_c1", "workload_c2", "workload_c3", "workload_c4",
    "workload_c5",
]


@dataclass
class CSR:
    """Canonical CSR matrix (sorted, duplicate-free columns)."""
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        return self.scipy().toarray()


def to_csr(m) -> CSR:
    """Convert any scipy sparse matrix to canonical CSR."""
    m = sp.csr_matrix(m, dtype=np.float64)
    m.sum_duplicates()
    m.sort_indices()
    return CSR(m.shape[0], m.indptr.astype(np.int64), m.indices.astype(np.int32),
               m.data.astype(np.float64))


def _lap1d(g: int) -> sp.csr_matrix:
    return sp.diags([np.ones(g - 1), -2.0 * np.ones(g), np.ones(g - 1)], [-1, 0, 1],
                    format="csr")


def laplacian_2d(g: int, scale: float = 1.0) -> CSR:
    """5-point Dirichlet Laplacian on a g x g interior grid, times ``scale``
    (diagonal -4*scale, neighbours +scale); row index = ix*g + iy."""
    i = sp.identity(g, format="csr")
    a = sp.kron(_lap1d(g), i) + sp.kron(i, _lap1d(g))
    return to_csr(a * scale)


def laplacian_3d(g: int, scale: float = 1.0) -> CSR:
    """7-point Dirichlet Laplacian on a g^3 interior grid, times ``scale``."""
    i = sp.identity(g, format="csr")
    l1 = _lap1d(g)
    a = (sp.kron(sp.kron(l1, i), i) + sp.kron(sp.kron(i, l1), i)
         + sp.kron(sp.kron(i, i), l1))
    return to_csr(a * scale)


def convdiff_3d(g: int, delta: float = 4.0, kappa: float = 1.0,
                b=(-1.0, -1.0, -1.0), speed: float = 1.25) -> CSR:
    """7-point upwind convection-diffusion operator kappa*Lap(u) + b.grad(u)
    on the interior g^3 grid of [-delta, delta]^3 (spacing h = 2 delta/(g+1)),
    Dirichlet zero boundary.  ``b`` is normalised to length ``speed``.

    Upwinding keeps every off-diagonal entry >= 0: for velocity component
    b_k the forward (b_k > 0) or backward (b_k < 0) neighbour gets |b_k|/h on
    top of kappa/h^2, and the diagonal gets -(6 kappa/h^2 + sum_k |b_k|/h)."""
    h = 2.0 * delta / (g + 1)
    bv = np.asarray(b, dtype=np.float64)
    bv = bv / np.linalg.norm(bv) * speed
    n = g ** 3
    idx = np.arange(n).reshape(g, g, g)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [
        np.full(n, -(6.0 * kappa / h ** 2 + np.abs(bv).sum() / h))]
    for axis in range(3):
        for step in (-1, 1):
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if step == 1:
                src[axis], dst[axis] = slice(0, g - 1), slice(1, g)
            else:
                src[axis], dst[axis] = slice(1, g), slice(0, g - 1)
            r = idx[tuple(src)].ravel()
            c = idx[tuple(dst)].ravel()
            upwind = abs(bv[axis]) / h if np.sign(bv[axis]) == step else 0.0
            rows.append(r)
            cols.append(c)
            vals.append(np.full(r.size, kappa / h ** 2 + upwind))
    a = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return to_csr(a)


def ba_graph(n: int, m: int, seed: int) -> CSR:
    """Symmetric 0/1 adjacency of a Barabasi-Albert graph: an (m+1)-clique
    seed, then every new node links to m distinct earlier nodes drawn with
    probability proportional to their degree (uniform draw from the list of
    edge endpoints).  No self-loops, no multi-edges."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    n_edges = m0 * (m0 - 1) // 2 + (n - m0) * m
    src = np.empty(n_edges, dtype=np.int64)
    dst = np.empty(n_edges, dtype=np.int64)
    ends = np.empty(2 * n_edges, dtype=np.int64)
    e = 0
    for a in range(m0):
        for b2 in range(a + 1, m0):
            src[e], dst[e] = a, b2
            ends[2 * e], ends[2 * e + 1] = a, b2
            e += 1
    ends_list = ends  # filled prefix [0, 2e) is the endpoint list
    block = 1 << 20
    u = rng.random(block)
    ui = 0
    for v in range(m0, n):
        pool = 2 * e
        chosen = set()
        while len(chosen) < m:
            if ui == block:
                u = rng.random(block)
                ui = 0
            chosen.add(int(ends_list[int(u[ui] * pool)]))
            ui += 1
        for t in sorted(chosen):
            src[e], dst[e] = v, t
            ends_list[2 * e], ends_list[2 * e + 1] = v, t
            e += 1
    ones = np.ones(2 * n_edges)
    a = sp.csr_matrix((ones, (np.concatenate([src, dst]), np.concatenate([dst, src]))),
                      shape=(n, n))
    return to_csr(a)


def small_world(n: int, k: int, p: float, seed: int) -> CSR:
    """Symmetric 0/1 adjacency of a Newman-Watts small-world network: a ring
    on which every node links to its k nearest neighbours on each side, plus,
    for each of the n k ring edges independently with probability p, a
    shortcut from the edge's first node to a node drawn uniformly from the
    other n - 1.  Shortcuts that repeat an existing edge are merged (0/1
    entries); there are no self-loops.  Stands in for the paper's small-world
    test networks (Sec. 4-5)."""
    if n < 2 * k + 2:
        raise ValueError("need n >= 2k + 2")
    rng = np.random.default_rng(seed)
    i = np.repeat(np.arange(n, dtype=np.int64), k)
    m = np.tile(np.arange(1, k + 1, dtype=np.int64), n)
    ring_dst = (i + m) % n
    take = rng.random(n * k) < p
    u = rng.integers(0, n - 1, size=n * k)
    short_dst = np.where(u >= i, u + 1, u)      # uniform over the other n - 1 nodes
    src = np.concatenate([i, i[take]])
    dst = np.concatenate([ring_dst, short_dst[take]])
    r = np.concatenate([src, dst])
    c = np.concatenate([dst, src])
    a = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(n, n))
    a.sum_duplicates()
    a.data[:] = 1.0
    return to_csr(a)


def random_sparse(n: int, per_row: int, seed: int, signed: bool = True,
                  diag: bool = True, scale: float = 1.0) -> CSR:
    """Random sparse matrix with about ``per_row`` off-diagonal entries per
    row, magnitudes in [0.1, 1)*scale, random signs when ``signed``, and a
    random diagonal in [-1, 1)*scale when ``diag``."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        k = int(rng.integers(0, 2 * per_row + 1)) if n > 1 else 0
        c = rng.choice(n, size=min(k, n), replace=False) if k else np.empty(0, np.int64)
        c = c[c != i]
        mag = rng.uniform(0.1, 1.0, size=c.size) * scale
        sgn = np.where(rng.random(c.size) < 0.5, -1.0, 1.0) if signed else 1.0
        rows.append(np.full(c.size, i))
        cols.append(c)
        vals.append(mag * sgn)
        if diag:
            rows.append(np.array([i]))
            cols.append(np.array([i]))
            vals.append(np.array([rng.uniform(-1.0, 1.0) * scale]))
    a = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return to_csr(a)


def star_graph(leaves: int, weight: float = 1.0) -> CSR:
    """Adjacency of a star: node 0 linked to nodes 1..leaves (so node 0 has
    degree ``leaves`` and every leaf degree 1)."""
    n = leaves + 1
    r = np.concatenate([np.zeros(leaves, np.int64), np.arange(1, n)])
    c = np.concatenate([np.arange(1, n), np.zeros(leaves, np.int64)])
    a = sp.csr_matrix((np.full(2 * leaves, weight), (r, c)), shape=(n, n))
    return to_csr(a)


def ring_graph(n: int) -> CSR:
    """Adjacency of a cycle on n >= 3 nodes (every degree 2)."""
    i = np.arange(n)
    r = np.concatenate([i, i])
    c = np.concatenate([(i + 1) % n, (i - 1) % n])
    return to_csr(sp.csr_matrix((np.ones(2 * n), (r, c)), shape=(n, n)))


def lambda_max(a: CSR, tol: float = 1e-12, max_iter: int = 100000, seed: int = 7) -> float:
    """Largest eigenvalue of a symmetric nonnegative matrix by power
    iteration, stopped when the Rayleigh quotient changes by < tol
    (relative)."""
    m = a.scipy()
    x = np.random.default_rng(seed).random(a.n) + 0.5
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(max_iter):
        y = m @ x
        new = float(x @ y)
        ny = np.linalg.norm(y)
        if ny == 0.0:
            return 0.0
        x = y / ny
        if abs(new - lam) <= tol * abs(new):
            return new
        lam = new
    return lam


def uniform_v(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform in [0, 1)."""
    return np.random.default_rng(seed).random(n)


@dataclass
class Workload:
    """One synthetic problem: x = exp(t A) v to relative tolerance ``tol``."""
    name: str
    a: CSR
    t: float
    v: np.ndarray
    tol: float
    num_levels: int
    precision: str  # "fp64" or "fp32"
    extra: dict = field(default_factory=dict)


def workload_c1(seed: int = 20190429) -> Workload:
    """2D 5-point Dirichlet Laplacian on a 32x32 grid scaled by 1/h^2
    (h = 1/33), t with t*||A||_inf = 4, v uniform [0,1); 3 levels, rel. RMS
    1e-2, FP64 walks."""
    g = 32
    h = 1.0 / (g + 1)
    a = laplacian_2d(g, 1.0 / h ** 2)
    t = 4.0 / (8.0 / h ** 2)
    return Workload("laplace2d_32x32_fp64", a, t, uniform_v(a.n, seed + 0), 1e-2, 3, "fp64",
                    {"grid": g, "h": h})


def workload_c2(seed: int = 20190429, n: int = 100_000, m: int = 4) -> Workload:
    """Total communicability of a Barabasi-Albert graph (n=1e5, m=4),
    beta = 1/lambda_max by power iteration, v = 1; 4 levels, rel. error
    1e-3, FP32 walk weights with FP64 final sum."""
    a = ba_graph(n, m, seed + 1)
    lam = lambda_max(a)
    return Workload(f"ba_n{n}_m{m}_tc_fp32", a, 1.0 / lam, np.ones(a.n), 1e-3, 4, "fp32",
                    {"lambda_max": lam, "d_max": float(np.diff(a.row_ptr).max())})


def workload_c3(seed: int = 20190429, count: int = 256, n_lo: float = 1e3,
                n_hi: float = 1e6) -> list:
    """Batch of independent unscaled integer-stencil Laplacians: n
    log-uniform in [n_lo, n_hi], half 2D (g = round(sqrt n)), half 3D
    (g = round(cbrt n)); t uniform in [0.1, 2]; 1-8 right-hand sides uniform
    in [0,1).  Returns a list of (Workload, rhs matrix [k, n])."""
    rng = np.random.default_rng(seed + 3)
    out = []
    for k in range(count):
        n = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        if k % 2 == 0:
            g = max(2, int(round(math.sqrt(n))))
            a = laplacian_2d(g)
        else:
            g = max(2, int(round(n ** (1.0 / 3.0))))
            a = laplacian_3d(g)
        t = float(rng.uniform(0.1, 2.0))
        nrhs = int(rng.integers(1, 9))
        rhs = rng.random((nrhs, a.n))
        out.append((Workload(f"batch{k}_{'2d' if k % 2 == 0 else '3d'}_g{g}", a, t, rhs[0],
                             1e-3, 3, "fp32"), rhs))
    return out


def workload_c4(seed: int = 20190429, g: int = 128) -> Workload:
    """3D upwind convection-diffusion on a g^3 interior grid of [-4,4]^3,
    kappa = 1, |b| = 1.25 along -(1,1,1)/sqrt3 (Peclet |b| 2 delta/kappa =
    10), t with t*||A||_inf = 8, v = exp(-|x|^2) (the paper's bump)."""
    delta = 4.0
    a = convdiff_3d(g, delta=delta, kappa=1.0, b=(-1.0, -1.0, -1.0), speed=1.25)
    h = 2.0 * delta / (g + 1)
    norm_inf = float(np.abs(a.scipy()).sum(axis=1).max())
    xs = -delta + h * np.arange(1, g + 1)
    x, y, z = np.meshgrid(xs, xs, xs, indexing="ij")
    v = np.exp(-(x ** 2 + y ** 2 + z ** 2)).ravel()
    return Workload(f"convdiff3d_{g}^3_fp32", a, 8.0 / norm_inf, v, 1e-3, 4, "fp32",
                    {"h": h, "norm_inf": norm_inf, "seed": seed})


def workload_c5(seed: int = 20190429, n: int = 1_000_000, m: int = 8) -> Workload:
    """Total communicability of a Barabasi-Albert graph (n=1e6, m=8),
    beta = 1/lambda_max, v = 1; rel. error 1e-3."""
    a = ba_graph(n, m, seed + 5)
    lam = lambda_max(a)
    return Workload(f"ba_n{n}_m{m}_tc", a, 1.0 / lam, np.ones(a.n), 1e-3, 4, "fp32",
                    {"lambda_max": lam})
