"""ctypes binding to the oracle's C walker (``mlmc_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The C file is compiled by :func:`build` with ``-ffp-contract=off`` so that
every floating-point operation rounds exactly as written; the GPU library
makes the same operations with explicit round-to-nearest intrinsics, which is
what lets index trajectories be compared bit for bit.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlmc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liborc_mlmc.so")
_lib = None

RESIDUAL, REDRAW, LITERAL_RATE = 0, 2, 3
FP64, FP32 = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class WalkRec(ct.Structure):
    _fields_ = [("end", ct.c_int32), ("jumps", ct.c_int32), ("sign", ct.c_int32),
                ("hash", ct.c_uint32), ("y", ct.c_double), ("y_alg2", ct.c_double),
                ("log_f", ct.c_double), ("log_c", ct.c_double), ("status", ct.c_int32),
                ("pad", ct.c_int32), ("src", ct.c_double), ("src_abs", ct.c_double)]


WALK_DTYPE = np.dtype([("end", np.int32), ("jumps", np.int32), ("sign", np.int32),
                       ("hash", np.uint32), ("y", np.float64), ("y_alg2", np.float64),
                       ("log_f", np.float64), ("log_c", np.float64), ("status", np.int32),
                       ("pad", np.int32), ("src", np.float64), ("src_abs", np.float64)])
assert WALK_DTYPE.itemsize == ct.sizeof(WalkRec)


class Ctx(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("row_ptr", ct.c_void_p), ("deg", ct.c_void_p),
                ("dl", ct.c_void_p), ("inv_rate", ct.c_void_p), ("inv_rate32", ct.c_void_p),
                ("thr", ct.c_void_p), ("keep_col", ct.c_void_p), ("keep_neg", ct.c_void_p),
                ("alias_col", ct.c_void_p), ("alias_neg", ct.c_void_p), ("v", ct.c_void_p),
                ("lr_keep", ct.c_void_p), ("lr_alias", ct.c_void_p), ("seed", ct.c_uint64),
                ("precision", ct.c_int32), ("variant", ct.c_int32), ("max_jumps", ct.c_int64),
                ("f", ct.c_void_p), ("t", ct.c_double), ("pieces", ct.c_int32),
                ("pad_pieces", ct.c_int32)]


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        P = ct.c_void_p
        _lib.orc_philox4x32_10.argtypes = [P, P, P]
        _lib.orc_uniform64.argtypes = [ct.c_uint32, ct.c_uint32]
        _lib.orc_uniform64.restype = ct.c_double
        _lib.orc_uniform32.argtypes = [ct.c_uint32]
        _lib.orc_uniform32.restype = ct.c_float
        _lib.orc_neglog64.argtypes = [ct.c_double]
        _lib.orc_neglog64.restype = ct.c_double
        _lib.orc_neglog32.argtypes = [ct.c_float]
        _lib.orc_neglog32.restype = ct.c_float
        _lib.orc_neglog64_batch.argtypes = [P, P, ct.c_int64]
        _lib.orc_neglog32_batch.argtypes = [P, P, ct.c_int64]
        _lib.orc_split.argtypes = [ct.c_int64, P, P, P, ct.c_double, P, P, P, P, P, P, P]
        _lib.orc_alias.argtypes = [ct.c_int64, P, P, P, P, P, P, P, P, P, P]
        _lib.orc_alias.restype = ct.c_int
        _lib.orc_alias_is.argtypes = [ct.c_int64, P, P, P, P, P, P, ct.c_double, P, P, P, P, P, P,
                                      P]
        _lib.orc_alias_is.restype = ct.c_int
        _lib.orc_walk_times_many.argtypes = [P, ct.c_int64, P, P, ct.c_int, ct.c_int, ct.c_int32,
                                             P, P]
        _lib.orc_walk_times_many.restype = ct.c_int
        _lib.orc_tilt_rates.argtypes = [ct.c_int64, P, P, P, P, P, ct.c_double, P]
        _lib.orc_tilt_rates.restype = ct.c_int
        _lib.orc_tilted_split.argtypes = [ct.c_int64, ct.c_double, P, P, P, P, P, P]
        _lib.orc_tilted_split.restype = ct.c_int
        _lib.orc_alias_tilt.argtypes = [ct.c_int64, P, P, P, P, P, P, ct.c_double, P, P, P, P, P,
                                        P, P, P]
        _lib.orc_alias_tilt.restype = ct.c_int
        _lib.orc_walk.argtypes = [ct.POINTER(Ctx), ct.c_int64, ct.c_int64, ct.c_int, ct.c_int,
                                  ct.POINTER(WalkRec)]
        _lib.orc_walk_many.argtypes = [ct.POINTER(Ctx), ct.c_int64, P, P, ct.c_int, ct.c_int, P]
        _lib.orc_mlmcl.argtypes = [ct.POINTER(Ctx), ct.c_int64, ct.c_int64, ct.c_int64,
                                   ct.c_int64, ct.c_int, ct.c_int, ct.c_int, P, P, P, P]
        _lib.orc_max_threads.restype = ct.c_int
        _lib.orc_walk_fwd_many.argtypes = [ct.POINTER(Ctx), P, P, ct.c_uint64, ct.c_uint64,
                                           ct.c_int64, ct.c_int, ct.c_int, P]
        _lib.orc_mlmcl_fwd.argtypes = [ct.POINTER(Ctx), P, P, ct.c_uint64, ct.c_uint64, ct.c_int64,
                                       ct.c_int, ct.c_int, P, P, P, P]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x uint32) under one key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def neglog64(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    lib().orc_neglog64_batch(_p(u), _p(out), u.size)
    return out


def neglog32(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty_like(u)
    lib().orc_neglog32_batch(_p(u), _p(out), u.size)
    return out


@dataclass
class Tables:
    """The oracle's per-row split quantities and alias tables."""
    n: int
    row_ptr: np.ndarray
    a_ii: np.ndarray
    L: np.ndarray
    deg: np.ndarray
    dl: np.ndarray
    inv_rate: np.ndarray
    inv_rate32: np.ndarray
    dl32: np.ndarray
    thr: np.ndarray
    keep_col: np.ndarray
    keep_neg: np.ndarray
    alias_col: np.ndarray
    alias_neg: np.ndarray
    lr_keep: np.ndarray = None   # proposal tables only: log(k/q) of the kept column
    lr_alias: np.ndarray = None  # ... and of the alias column
    lam: np.ndarray = None       # tilted clocks only: the walk's rates lambda_i
    pieces: int = 1              # R19 time pieces: per-row arrays hold `pieces` blocks of n,
                                 # entry arrays `pieces` blocks of nnz (build_tables_pieces)


def build_tables(a, t: float, h=None, alpha: float = 0.1, clocks: bool = False) -> Tables:
    """Splitting (Eq. 1) and alias tables (Eq. 12) of the CSR matrix ``a``
    for time ``t``.  ``a`` has fields n, row_ptr, col, val.  With ``h`` (n
    positive float32 values) the tables sample the importance-sampling
    proposal q = (1-alpha) |a_ij| h_j / sum + alpha k_ij instead, and record
    log(k/q) per entry.  With ``clocks`` as well, the holding times are
    tilted too (the h-transform, orc_tilt_rates): the walk's rates are
    lambda_i = sum_j |a_ij| h_j / h_i (clamped to [L_ii/1024, max(L_ii, 2/t)]),
    dl_i = t (a_ii + lambda_i), and every entry of row i also records
    log(L_ii / lambda_i)."""
    n = a.n
    rp = np.ascontiguousarray(a.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(a.col, dtype=np.int32)
    val = np.ascontiguousarray(a.val, dtype=np.float64)
    nnz = int(rp[-1])
    a_ii = np.zeros(n)
    L = np.zeros(n)
    deg = np.zeros(n, dtype=np.int32)
    dl = np.zeros(n)
    inv_rate = np.zeros(n)
    inv_rate32 = np.zeros(n, dtype=np.float32)
    dl32 = np.zeros(n, dtype=np.float32)
    lib().orc_split(n, _p(rp), _p(col), _p(val), float(t), _p(a_ii), _p(L), _p(deg), _p(dl),
                    _p(inv_rate), _p(inv_rate32), _p(dl32))
    m = max(nnz, 1)
    thr = np.zeros(m, dtype=np.uint32)
    keep_col = np.full(m, -1, dtype=np.int32)
    keep_neg = np.zeros(m, dtype=np.uint8)
    alias_col = np.full(m, -1, dtype=np.int32)
    alias_neg = np.zeros(m, dtype=np.uint8)
    lam = None
    if h is None:
        if clocks:
            raise ValueError("tilted clocks need h")
        rc = lib().orc_alias(n, _p(rp), _p(col), _p(val), _p(L), _p(deg), _p(thr), _p(keep_col),
                             _p(keep_neg), _p(alias_col), _p(alias_neg))
        lr_keep = lr_alias = None
    elif clocks:
        hh = np.ascontiguousarray(h, dtype=np.float32)
        lam = np.zeros(n)
        lib().orc_tilt_rates(n, _p(rp), _p(col), _p(val), _p(L), _p(hh), float(t), _p(lam))
        lib().orc_tilted_split(n, float(t), _p(a_ii), _p(lam), _p(dl), _p(inv_rate),
                               _p(inv_rate32), _p(dl32))
        lr_keep = np.zeros(m, dtype=np.float32)
        lr_alias = np.zeros(m, dtype=np.float32)
        rc = lib().orc_alias_tilt(n, _p(rp), _p(col), _p(val), _p(L), _p(deg), _p(hh),
                                  float(alpha), _p(lam), _p(thr), _p(keep_col), _p(keep_neg),
                                  _p(alias_col), _p(alias_neg), _p(lr_keep), _p(lr_alias))
    else:
        hh = np.ascontiguousarray(h, dtype=np.float32)
        lr_keep = np.zeros(m, dtype=np.float32)
        lr_alias = np.zeros(m, dtype=np.float32)
        rc = lib().orc_alias_is(n, _p(rp), _p(col), _p(val), _p(L), _p(deg), _p(hh), float(alpha),
                                _p(thr), _p(keep_col), _p(keep_neg), _p(alias_col),
                                _p(alias_neg), _p(lr_keep), _p(lr_alias))
    if rc != 0:
        raise MemoryError("oracle alias build failed")
    return Tables(n, rp, a_ii, L, deg, dl, inv_rate, inv_rate32, dl32, thr, keep_col, keep_neg,
                  alias_col, alias_neg, lr_keep, lr_alias, lam)


def build_tables_pieces(a, t: float, hs, alpha: float = 0.1) -> Tables:
    """Tilted-clock tables of a proposal that changes with time (reading
    R19): ``hs`` holds K rows of h, row p for the piece [p/K, (p+1)/K) of
    scaled time; piece p's tables are build_tables(a, t, hs[p], alpha,
    clocks=True), stacked piece after piece."""
    hs = np.asarray(hs, dtype=np.float32)
    if hs.ndim != 2 or hs.shape[0] < 1:
        raise ValueError("hs: K rows of n values")
    parts = [build_tables(a, t, hs[p], alpha, clocks=True) for p in range(hs.shape[0])]
    if len(parts) == 1:
        return parts[0]
    b0 = parts[0]
    cat = lambda name: np.ascontiguousarray(np.concatenate([getattr(q, name) for q in parts]))
    return Tables(b0.n, b0.row_ptr, b0.a_ii, b0.L, b0.deg, cat("dl"), cat("inv_rate"),
                  cat("inv_rate32"), cat("dl32"), cat("thr"), cat("keep_col"), cat("keep_neg"),
                  cat("alias_col"), cat("alias_neg"), cat("lr_keep"), cat("lr_alias"), cat("lam"),
                  len(parts))


class Walker:
    """Replays walks of Algorithm 2 on one matrix, time and right-hand side."""

    def __init__(self, a, t: float, v: np.ndarray, seed: int, precision: int = FP64,
                 variant: int = RESIDUAL, max_jumps: int = 1 << 30, tables: Tables = None,
                 f: np.ndarray = None):
        """f: the constant source vector of Algorithm 3 (None: no source term);
        with it every walk also carries its Simpson source part (record field
        `src`), and mlmcl sums y + src."""
        self.tables = tables if tables is not None else build_tables(a, t)
        self.v = np.ascontiguousarray(v, dtype=np.float64)
        self.f = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
        tb = self.tables
        self._keep = (tb, self.v, self.f)
        lrk = _p(tb.lr_keep).value if tb.lr_keep is not None else None
        lra = _p(tb.lr_alias).value if tb.lr_alias is not None else None
        self.ctx = Ctx(tb.n, _p(tb.row_ptr).value, _p(tb.deg).value, _p(tb.dl).value,
                       _p(tb.inv_rate).value, _p(tb.inv_rate32).value, _p(tb.thr).value,
                       _p(tb.keep_col).value, _p(tb.keep_neg).value, _p(tb.alias_col).value,
                       _p(tb.alias_neg).value, _p(self.v).value, lrk, lra, ct.c_uint64(seed),
                       precision, variant, max_jumps,
                       _p(self.f).value if self.f is not None else None, float(t),
                       tb.pieces, 0)

    def walk(self, row: int, rep: int, level: int, coarse: bool) -> WalkRec:
        r = WalkRec()
        lib().orc_walk(ct.byref(self.ctx), row, rep, level, int(coarse), ct.byref(r))
        return r

    def walks_times(self, rows, reps, level: int, coarse: bool, n_times: int):
        """walks() plus each walk's samples of the intermediate times t k /
        n_times, k = 1..n_times-1 (array [count, n_times-1])."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        reps = np.ascontiguousarray(reps, dtype=np.int64)
        out = np.zeros(rows.size, dtype=WALK_DTYPE)
        yt = np.zeros((rows.size, n_times - 1))
        lib().orc_walk_times_many(ct.byref(self.ctx), rows.size, _p(rows), _p(reps), level,
                                  int(coarse), n_times, _p(out), _p(yt))
        return out, yt

    def walks(self, rows, reps, level: int, coarse: bool) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        reps = np.ascontiguousarray(reps, dtype=np.int64)
        out = np.zeros(rows.size, dtype=WALK_DTYPE)
        lib().orc_walk_many(ct.byref(self.ctx), rows.size, _p(rows), _p(reps), level,
                            int(coarse), _p(out))
        return out

    def mlmcl(self, level: int, coarse: bool, rep_begin: int, reps: int, rows=None,
              nthreads: int = 0):
        """Algorithm 2 over rows [r0, r1) x replicas [rep_begin, rep_begin+reps):
        returns (per-row sum of y, total sum of y^2, total jumps, limit hits)."""
        r0, r1 = (0, self.tables.n) if rows is None else rows
        sum_y = np.zeros(self.tables.n)
        sum_y2 = np.zeros(1)
        jumps = np.zeros(1, dtype=np.int64)
        lim = np.zeros(1, dtype=np.int64)
        lib().orc_mlmcl(ct.byref(self.ctx), r0, r1, rep_begin, reps, level, int(coarse),
                        nthreads, _p(sum_y), _p(sum_y2), _p(jumps), _p(lim))
        return sum_y, float(sum_y2[0]), int(jumps[0]), int(lim[0])


def max_threads() -> int:
    return int(lib().orc_max_threads())


def transpose(a):
    """Canonical CSR of A^T (forward mode walks on it)."""
    import scipy.sparse as sp
    m = sp.csr_matrix((a.val, a.col, a.row_ptr), shape=(a.n, a.n)).T.tocsr()
    m.sort_indices()
    from types import SimpleNamespace
    return SimpleNamespace(n=a.n, row_ptr=m.indptr.astype(np.int64), col=m.indices.astype(np.int32),
                           val=m.data.astype(np.float64))


def start_weights(v: np.ndarray):
    """Integer start weights w_s = ceil(|v_s|/max|v| * 2^20) (0 where v_s = 0),
    their inclusive prefix sums and total (exact integer arithmetic)."""
    av = np.abs(np.asarray(v, dtype=np.float64))
    vmax = av.max()
    w = np.where(av > 0, np.ceil((av / vmax) * 1048576.0), 0).astype(np.int64)
    cdf = np.cumsum(w).astype(np.int64)
    return w, cdf, int(cdf[-1])


class ForwardWalker(Walker):
    """Forward-mode walks (Eq. 5): tables of A^T, starts drawn ~ |v|."""

    def __init__(self, a, t: float, v: np.ndarray, seed: int, precision: int = FP64,
                 max_jumps: int = 1 << 30, h=None, alpha: float = 0.1, clocks: bool = False):
        b = transpose(a)
        tables = build_tables(b, t, h, alpha, clocks) if h is not None else build_tables(b, t)
        super().__init__(b, t, v, seed, precision=precision, max_jumps=max_jumps, tables=tables)
        self.w, self.cdf, self.W = start_weights(v)

    def walks_fwd(self, g0: int, count: int, level: int, coarse: bool) -> np.ndarray:
        out = np.zeros(count, dtype=WALK_DTYPE)
        lib().orc_walk_fwd_many(ct.byref(self.ctx), _p(self.cdf), _p(self.w), ct.c_uint64(self.W),
                                ct.c_uint64(g0), count, level, int(coarse), _p(out))
        return out

    def mlmcl_fwd(self, level: int, coarse: bool, g0: int, count: int):
        sum_x = np.zeros(self.tables.n)
        sum_y2 = np.zeros(1)
        jumps = np.zeros(1, dtype=np.int64)
        lim = np.zeros(1, dtype=np.int64)
        lib().orc_mlmcl_fwd(ct.byref(self.ctx), _p(self.cdf), _p(self.w), ct.c_uint64(self.W),
                            ct.c_uint64(g0), count, level, int(coarse), _p(sum_x), _p(sum_y2),
                            _p(jumps), _p(lim))
        return sum_x, float(sum_y2[0]), int(jumps[0]), int(lim[0])
