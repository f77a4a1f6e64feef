"""Thin Python binding of libmlmc (``include/mlmc.h``): argument marshalling
only.  Every step of the estimator runs in the library's CUDA kernels; there
is no CPU fallback, and loading fails loudly when the library is missing.

Arrays may be numpy arrays (host memory) or torch tensors (host or device);
the library copies host/device data through unified addressing.  Entry points
documented as device-only in the header take torch CUDA tensors.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

MLMC_OK, MLMC_ERR_INVALID_ARG, MLMC_ERR_CUDA, MLMC_ERR_OOM = 0, 1, 2, 3
MLMC_ERR_NOT_CONVERGED, MLMC_ERR_WALK_LIMIT, MLMC_ERR_NUMERIC = 4, 5, 6
MLMC_ERR_EXCHANGE = 7
FP64, FP32_KAHAN = 0, 1
BACKWARD, FORWARD = 0, 1
PLAIN, LEARNED = 0, 1
TILT_JUMPS, TILT_CLOCKS, TILT_TIME = 1, 2, 4

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED",
           5: "WALK_LIMIT", 6: "NUMERIC", 7: "EXCHANGE"}


class MlmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mlmc {_STATUS.get(status, status)}: {msg}")
        self.status = status


# int32_t (*mlmc_exchange_fn)(int64_t count, void *ctx)
EXCHANGE_FN = ct.CFUNCTYPE(ct.c_int32, ct.c_int64, ct.c_void_p)


class Schedule(ct.Structure):
    _fields_ = [("l0", ct.c_int32), ("num_levels", ct.c_int32), ("max_levels", ct.c_int32),
                ("precision", ct.c_int32), ("mode", ct.c_int32), ("proposal", ct.c_int32),
                ("pilot_walks", ct.c_int64), ("max_jumps_per_walk", ct.c_int64),
                ("max_walks_per_row", ct.c_int64), ("time_budget_s", ct.c_double),
                ("walks_per_lane", ct.c_int32), ("block_threads", ct.c_int32),
                ("l2_persist", ct.c_int32), ("launch_reps", ct.c_int32)]


class LevelStats(ct.Structure):
    _fields_ = [("level", ct.c_int32), ("pad", ct.c_int32), ("walks_per_row", ct.c_int64),
                ("mean_norm2", ct.c_double), ("var", ct.c_double),
                ("cost_events_per_walk", ct.c_double), ("jumps", ct.c_int64),
                ("seconds", ct.c_double), ("launches", ct.c_int64), ("still_walks", ct.c_int64)]


WALK_RECORD_DTYPE = np.dtype([("end", np.int32), ("jumps", np.int32), ("sign", np.int32),
                              ("hash", np.uint32), ("y", np.float64), ("status", np.int32),
                              ("pad", np.int32)])

_lib = None


def _checked() -> bool:
    return os.environ.get("MLMC_CHECKED", "0") == "1"


def library_path() -> str:
    """The library this process loads: libmlmc.so, or the checked build
    libmlmc_checked.so when the environment sets MLMC_CHECKED=1."""
    return _build.LIB_CHECKED if _checked() else _build.LIB


def load(build_if_missing: bool = False):
    """Load libmlmc.so (building it first if asked; the checked build is
    always built on demand).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not (build_if_missing or _checked()):
            raise ImportError(f"libmlmc.so not built ({path}); run __graft_entry__.build()")
        _build.build(checked=_checked())
    lib = ct.CDLL(path)
    P, I64, I32, D = ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_double
    lib.mlmc_schedule_default.argtypes = [ct.POINTER(Schedule)]
    lib.mlmc_plan_create.argtypes = [ct.POINTER(P), I64, I64, P, P, P, D, ct.POINTER(Schedule),
                                     D, P]
    lib.mlmc_plan_rebuild.argtypes = [P]
    lib.mlmc_expmv.argtypes = [P, P, P, ct.c_uint64]
    lib.mlmc_stats.argtypes = [P, P, I32, ct.POINTER(I32), ct.POINTER(D)]
    lib.mlmc_expmv_entry.argtypes = [P, I64, P, ct.POINTER(D), ct.c_uint64]
    lib.mlmc_expmv_sum.argtypes = [P, P, ct.POINTER(D), ct.c_uint64]
    lib.mlmc_mlmcl.argtypes = [P, I32, I32, I64, I64, P, ct.c_uint64, P, P]
    lib.mlmc_trace.argtypes = [P, I32, I32, I64, I64, P, ct.c_uint64, P]
    lib.mlmc_trace_noalloc.argtypes = [P, I32, I32, I64, I64, P, ct.c_uint64, P]
    lib.mlmc_trace_times.argtypes = [P, I32, I32, I64, I64, P, ct.c_uint64, I32, P, P]
    lib.mlmc_expmv_times.argtypes = [P, P, P, I32, ct.c_uint64]
    lib.mlmc_export_tables.argtypes = [P] + [P] * 11
    lib.mlmc_plan_info.argtypes = [P, ct.POINTER(I64), ct.POINTER(I64), ct.POINTER(I32),
                                   ct.POINTER(D)]
    lib.mlmc_plan_destroy.argtypes = [P]
    lib.mlmc_plan_destroy.restype = None
    lib.mlmc_last_error.restype = ct.c_char_p
    lib.mlmc_batch_create.argtypes = [ct.POINTER(P), P, I32, ct.POINTER(Schedule), D, P]
    lib.mlmc_batch_expmv.argtypes = [P, P, P, P]
    lib.mlmc_batch_stats.argtypes = [P, I32, P, I32, ct.POINTER(I32), ct.POINTER(D)]
    lib.mlmc_batch_info.argtypes = [P, ct.POINTER(I64), ct.POINTER(D), ct.POINTER(I32)]
    lib.mlmc_batch_autotune.argtypes = [P, P, I32]
    lib.mlmc_batch_destroy.argtypes = [P]
    lib.mlmc_batch_destroy.restype = None
    lib.mlmc_plan_set_proposal.argtypes = [P, P, D]
    lib.mlmc_plan_set_tilt.argtypes = [P, P, D, I32]
    lib.mlmc_export_tilt.argtypes = [P] + [P] * 6
    lib.mlmc_plan_set_tilt_pieces.argtypes = [P, P, I32, D]
    lib.mlmc_plan_tilt_pieces.argtypes = [P]
    lib.mlmc_plan_tilt_pieces.restype = I32
    lib.mlmc_export_tilt_piece.argtypes = [P, I32] + [P] * 6
    lib.mlmc_export_proposal_piece.argtypes = [P, I32] + [P] * 7
    lib.mlmc_export_h.argtypes = [P, P]
    lib.mlmc_plan_learn_report.argtypes = [P, ct.POINTER(I32), P, I32, ct.POINTER(I32)]
    lib.mlmc_shard_buffer_doubles.argtypes = [P]
    lib.mlmc_shard_buffer_doubles.restype = I64
    lib.mlmc_shard_range.argtypes = [I64, I32, I32, ct.POINTER(I64), ct.POINTER(I64)]
    lib.mlmc_plan_set_shard.argtypes = [P, I32, I32, P, P, P, I64]  # the exchange as a void*
    lib.mlmc_plan_set_source.argtypes = [P, P]
    lib.mlmc_plan_l2_window.argtypes = [P, ct.POINTER(I64), ct.POINTER(D)]
    lib.mlmc_plan_save_state.argtypes = [P, P, ct.c_size_t, ct.POINTER(ct.c_size_t)]
    lib.mlmc_plan_load_state.argtypes = [P, P, ct.c_size_t]
    lib.mlmc_expmv_resume.argtypes = [P, P]
    lib.mlmc_export_proposal.argtypes = [P] + [P] * 7
    lib.mlmc_mlp_create.argtypes = [ct.POINTER(P), ct.c_uint64, P]
    lib.mlmc_mlp_destroy.argtypes = [P]
    lib.mlmc_mlp_destroy.restype = None
    lib.mlmc_mlp_param_count.restype = I32
    lib.mlmc_mlp_params.argtypes = [P, P, P]
    lib.mlmc_mlp_forward.argtypes = [P, P, I64, P]
    lib.mlmc_mlp_loss_grad.argtypes = [P, P, P, I64, P, P]
    lib.mlmc_mlp_train.argtypes = [P, P, P, I64, I32, I32, ct.c_float, ct.c_uint64, P]
    lib.mlmc_learn_proposal.argtypes = [P, P, P, ct.c_uint64, I64, I32, I32, ct.c_float, D, P]
    lib.mlmc_learn_tilt.argtypes = [P, P, P, ct.c_uint64, I64, I32, I32, ct.c_float, D, I32, I32,
                                    P]
    lib.mlmc_mlp_launch_count.argtypes = [P]
    lib.mlmc_mlp_launch_count.restype = I64
    lib.mlmc_launch_count.argtypes = [P]
    lib.mlmc_launch_count.restype = I64
    for name in ("mlmc_schedule_default", "mlmc_plan_create", "mlmc_plan_rebuild", "mlmc_expmv",
                 "mlmc_expmv_entry", "mlmc_expmv_sum",
                 "mlmc_stats", "mlmc_mlmcl", "mlmc_trace", "mlmc_trace_noalloc",
                 "mlmc_trace_times", "mlmc_expmv_times",
                 "mlmc_export_tables", "mlmc_batch_create", "mlmc_batch_expmv",
                 "mlmc_batch_stats", "mlmc_batch_info", "mlmc_batch_autotune",
                 "mlmc_plan_set_proposal", "mlmc_plan_set_tilt", "mlmc_export_tilt",
                 "mlmc_plan_set_tilt_pieces", "mlmc_export_tilt_piece", "mlmc_export_proposal_piece",
                 "mlmc_export_h", "mlmc_plan_learn_report", "mlmc_shard_range",
                 "mlmc_plan_set_shard",
                 "mlmc_plan_set_source", "mlmc_plan_l2_window",
                 "mlmc_plan_save_state", "mlmc_plan_load_state", "mlmc_expmv_resume",
                 "mlmc_export_proposal",
                 "mlmc_mlp_create",
                 "mlmc_mlp_params", "mlmc_mlp_forward", "mlmc_mlp_loss_grad", "mlmc_mlp_train",
                 "mlmc_learn_proposal", "mlmc_learn_tilt",
                 "mlmc_plan_info"):
        getattr(lib, name).restype = ct.c_int
    _lib = lib
    return lib


def _check(status: int, allow=()):
    if status != MLMC_OK and status not in allow:
        msg = _lib.mlmc_last_error().decode(errors="replace")
        raise MlmcError(status, msg)
    return status


def _nbytes(a) -> int:
    if isinstance(a, np.ndarray):
        return a.nbytes
    if hasattr(a, "element_size"):
        return a.numel() * a.element_size()
    return -1


def _need(a, nbytes: int, what: str):
    """Refuse a buffer smaller than the entry point will touch."""
    have = _nbytes(a)
    if have >= 0 and have < nbytes:
        raise ValueError(f"{what}: buffer of {have} bytes, need {nbytes}")


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"cannot take the address of {type(a)}")


def shard_range(extra: int, rank: int, world: int):
    """The walk indices [lo, hi) of `extra` new ones that rank `rank` of
    `world` takes in a sharded solve (mlmc_shard_range; no device work)."""
    lo, hi = ct.c_int64(), ct.c_int64()
    _check(load().mlmc_shard_range(int(extra), int(rank), int(world), ct.byref(lo), ct.byref(hi)))
    return lo.value, hi.value


def schedule_default(**overrides) -> Schedule:
    lib = load()
    s = Schedule()
    _check(lib.mlmc_schedule_default(ct.byref(s)))
    for k, v in overrides.items():
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    return s


class Plan:
    """An mlmc_plan: x = exp(t A) v for one CSR matrix A and time t."""

    def __init__(self, n: int, row_ptr, col, vals, t: float, sched: Schedule = None,
                 rel_tol: float = 1e-3, stream: int = 0):
        lib = load()
        self._lib = lib
        self._h = ct.c_void_p()
        nnz = int(row_ptr[-1]) if isinstance(row_ptr, np.ndarray) else int(row_ptr[-1].item())
        self._keep = (row_ptr, col, vals)
        _check(lib.mlmc_plan_create(ct.byref(self._h), int(n), nnz, _ptr(row_ptr), _ptr(col),
                                    _ptr(vals), float(t),
                                    ct.byref(sched) if sched is not None else None,
                                    float(rel_tol), ct.c_void_p(stream)))
        self.n, self.nnz = int(n), nnz
        self.mode = int(sched.mode) if sched is not None else BACKWARD

    def _trace_records(self, reps: int) -> int:
        # forward mode: one record per walk; backward: one per (row, rep)
        return reps if self.mode == FORWARD else self.n * reps

    @classmethod
    def from_csr(cls, a, t: float, sched: Schedule = None, rel_tol: float = 1e-3,
                 stream: int = 0):
        return cls(a.n, np.ascontiguousarray(a.row_ptr, np.int64),
                   np.ascontiguousarray(a.col, np.int32), np.ascontiguousarray(a.val, np.float64),
                   t, sched, rel_tol, stream)

    def close(self):
        if self._h:
            self._lib.mlmc_plan_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    def rebuild(self):
        _check(self._lib.mlmc_plan_rebuild(self._h))

    def expmv(self, v, x, seed: int, allow_not_converged: bool = False) -> int:
        _need(v, 8 * self.n, "v")
        _need(x, 8 * self.n, "x")
        allow = (MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        return _check(self._lib.mlmc_expmv(self._h, _ptr(v), _ptr(x), ct.c_uint64(seed)), allow)

    def expmv_times(self, v, x_times, n_times: int, seed: int,
                    allow_not_converged: bool = False) -> int:
        """x(t k / n_times), k = 1..n_times, from the same walks (x_times:
        n_times x n float64, host or device; the last row is x(t))."""
        _need(v, 8 * self.n, "v")
        _need(x_times, 8 * self.n * n_times, "x_times")
        allow = (MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        return _check(self._lib.mlmc_expmv_times(self._h, _ptr(v), _ptr(x_times), int(n_times),
                                                 ct.c_uint64(seed)), allow)

    def trace_times(self, level: int, coarse: bool, rep_begin: int, reps: int, v, seed: int,
                    n_times: int, rec, y_times):
        """trace() plus each record's samples at the times t k / n_times,
        k < n_times (y_times: device, n * reps * (n_times - 1) float64)."""
        _need(v, 8 * self.n, "v")
        _need(rec, WALK_RECORD_DTYPE.itemsize * self.n * reps, "rec")
        _need(y_times, 8 * self.n * reps * (n_times - 1), "y_times")
        _check(self._lib.mlmc_trace_times(self._h, level, int(coarse), rep_begin, reps, _ptr(v),
                                          ct.c_uint64(seed), int(n_times), _ptr(rec),
                                          _ptr(y_times)))

    def expmv_entry(self, i: int, v, seed: int, allow_not_converged: bool = False) -> float:
        """x_i = (exp(tA)v)_i by walks from row i only (Algorithm 2)."""
        _need(v, 8 * self.n, "v")
        out = ct.c_double()
        allow = (MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        _check(self._lib.mlmc_expmv_entry(self._h, int(i), _ptr(v), ct.byref(out),
                                          ct.c_uint64(seed)), allow)
        return out.value

    def expmv_sum(self, v, seed: int, allow_not_converged: bool = False) -> float:
        """1^T exp(tA) v (total communicability for v = 1)."""
        _need(v, 8 * self.n, "v")
        out = ct.c_double()
        allow = (MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        _check(self._lib.mlmc_expmv_sum(self._h, _ptr(v), ct.byref(out), ct.c_uint64(seed)),
               allow)
        return out.value

    def stats(self):
        cap = 32
        arr = (LevelStats * cap)()
        nl = ct.c_int32()
        err = ct.c_double()
        _check(self._lib.mlmc_stats(self._h, arr, cap, ct.byref(nl), ct.byref(err)))
        levels = [{f: getattr(arr[k], f) for f, _ in LevelStats._fields_ if f != "pad"}
                  for k in range(nl.value)]
        return levels, err.value

    def mlmcl(self, level: int, coarse: bool, rep_begin: int, reps: int, v, seed: int, sum_y,
              totals):
        _need(v, 8 * self.n, "v")
        _need(sum_y, 8 * self.n, "sum_y")
        _need(totals, 8 * 5, "totals")
        _check(self._lib.mlmc_mlmcl(self._h, level, int(coarse), rep_begin, reps, _ptr(v),
                                    ct.c_uint64(seed), _ptr(sum_y), _ptr(totals)))

    def trace(self, level: int, coarse: bool, rep_begin: int, reps: int, v, seed: int, rec):
        """Walk records: backward plans n*reps (row-major by row), forward
        plans reps (walk rep_begin + k at k, start state in `pad`)."""
        _need(v, 8 * self.n, "v")
        _need(rec, WALK_RECORD_DTYPE.itemsize * self._trace_records(reps), "rec")
        _check(self._lib.mlmc_trace(self._h, level, int(coarse), rep_begin, reps, _ptr(v),
                                    ct.c_uint64(seed), _ptr(rec)))

    def trace_noalloc(self, level: int, coarse: bool, rep_begin: int, reps: int, v, seed: int,
                      rec):
        """As trace(), through mlmc_trace_noalloc: no device allocation, the
        library's static scratch instead (at most 2^18 rows).  Asynchronous
        on the plan's stream."""
        _need(v, 8 * self.n, "v")
        _need(rec, WALK_RECORD_DTYPE.itemsize * self.n * reps, "rec")
        _check(self._lib.mlmc_trace_noalloc(self._h, level, int(coarse), rep_begin, reps,
                                            _ptr(v), ct.c_uint64(seed), _ptr(rec)))

    def export_tables(self) -> dict:
        n, nnz = self.n, self.nnz
        out = dict(l_ii=np.zeros(n), dl=np.zeros(n), inv_rate=np.zeros(n),
                   inv_rate32=np.zeros(n, np.float32), dl32=np.zeros(n, np.float32),
                   deg=np.zeros(n, np.int32), thr=np.zeros(max(nnz, 1), np.uint32),
                   keep_col=np.full(max(nnz, 1), -1, np.int32),
                   keep_neg=np.zeros(max(nnz, 1), np.uint8),
                   alias_col=np.full(max(nnz, 1), -1, np.int32),
                   alias_neg=np.zeros(max(nnz, 1), np.uint8))
        keys = ["l_ii", "dl", "inv_rate", "inv_rate32", "dl32", "deg", "thr", "keep_col",
                "keep_neg", "alias_col", "alias_neg"]
        _check(self._lib.mlmc_export_tables(self._h, *[_ptr(out[k]) for k in keys]))
        return out

    def set_source(self, f):
        """Constant source F of du/dt = A u + F (n float64 values, host or
        device; None removes it): later estimates return
        exp(tA) v + int_0^t exp(sA) F ds (Simpson's rule along the walks)."""
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
        elif f is not None and hasattr(f, "dtype") and str(f.dtype) != "torch.float64":
            raise TypeError("f must be float64")
        if f is not None:
            _need(f, 8 * self.n, "f")
        self._source = f
        _check(self._lib.mlmc_plan_set_source(self._h, _ptr(f)))

    def set_proposal(self, h, alpha: float = 0.1):
        """Importance-sampling jump proposal q ~ (1-alpha)|a_ij| h_j + alpha k_ij
        (h: n positive float32 values, host or device; None = plain law)."""
        if isinstance(h, np.ndarray):
            h = np.ascontiguousarray(h, dtype=np.float32)
        elif h is not None and hasattr(h, "dtype") and str(h.dtype) != "torch.float32":
            raise TypeError("h must be float32")
        if h is not None:
            _need(h, 4 * self.n, "h")
        _check(self._lib.mlmc_plan_set_proposal(self._h, _ptr(h) if h is not None else None,
                                                float(alpha)))

    def set_tilt(self, h, alpha: float = 0.1, clocks: bool = True):
        """Proposal with tilted jumps and, with ``clocks``, tilted holding
        times (the h-transform: rates sum_j |a_ij| h_j / h_i clamped to
        [L_ii/1024, max(L_ii, 2/t)]); h as in set_proposal (None = plain walk)."""
        if isinstance(h, np.ndarray):
            h = np.ascontiguousarray(h, dtype=np.float32)
        elif h is not None and hasattr(h, "dtype") and str(h.dtype) != "torch.float32":
            raise TypeError("h must be float32")
        if h is not None:
            _need(h, 4 * self.n, "h")
        tilt = TILT_JUMPS | (TILT_CLOCKS if clocks else 0)
        _check(self._lib.mlmc_plan_set_tilt(self._h, _ptr(h) if h is not None else None,
                                            float(alpha), tilt))

    def set_tilt_pieces(self, h, alpha: float = 0.1):
        """Tilted proposal with time pieces: h of shape (K, n) (numpy or a
        contiguous torch tensor), row p the h of the scaled times
        [p/K, (p+1)/K); None = plain walk."""
        if h is None:
            _check(self._lib.mlmc_plan_set_tilt_pieces(self._h, None, 1, float(alpha)))
            return
        if isinstance(h, np.ndarray):
            h = np.ascontiguousarray(h, dtype=np.float32)
        elif hasattr(h, "dtype") and str(h.dtype) != "torch.float32":
            raise TypeError("h must be float32")
        k = int(h.shape[0]) if len(h.shape) == 2 else 1
        if len(h.shape) == 2 and int(h.shape[1]) != self.n:
            raise ValueError("h: K rows of n values")
        _need(h, 4 * self.n * k, "h")
        _check(self._lib.mlmc_plan_set_tilt_pieces(self._h, _ptr(h), k, float(alpha)))

    def tilt_pieces(self) -> int:
        """Time pieces of the installed proposal (0 without one)."""
        return int(self._lib.mlmc_plan_tilt_pieces(self._h))

    def export_h(self) -> np.ndarray:
        """The h of the plan's proposal (float32, n; (K, n) with K > 1 time
        pieces)."""
        k = max(1, self.tilt_pieces())
        h = np.zeros(self.n * k, np.float32)
        _check(self._lib.mlmc_export_h(self._h, _ptr(h)))
        return h if k == 1 else h.reshape(k, self.n)

    def learn_report(self):
        """mlmc_plan_learn_report: (index of the installed law, per-walk
        variance at l0 of each pilot of the last learning)."""
        chosen, count = ct.c_int32(-1), ct.c_int32(0)
        var = np.zeros(16)
        _check(self._lib.mlmc_plan_learn_report(self._h, ct.byref(chosen), _ptr(var), 16,
                                                ct.byref(count)))
        return int(chosen.value), [float(x) for x in var[:min(count.value, 16)]]

    def shard_buffer_doubles(self) -> int:
        return int(self._lib.mlmc_shard_buffer_doubles(self._h))

    def set_shard(self, rank: int, world: int, exchange=None, buf=None):
        """Make the plan rank `rank` of a `world`-rank sharded solve.
        exchange: an EXCHANGE_FN (kept alive by the plan) that sums
        buf[0:count] over the ranks in place; buf: the exchange buffer (host
        or device, float64, at least shard_buffer_doubles()).  world = 1 or
        exchange = None: unsharded."""
        self._exchange = (exchange, buf)
        if exchange is None or world == 1:
            _check(self._lib.mlmc_plan_set_shard(self._h, 0, 1, None, None, None, 0))
            return
        _need(buf, 8 * self.shard_buffer_doubles(), "exchange buffer")
        cap = (buf.numel() if hasattr(buf, "numel") else buf.size)
        _check(self._lib.mlmc_plan_set_shard(self._h, int(rank), int(world),
                                             ct.cast(exchange, ct.c_void_p), None, _ptr(buf),
                                             int(cap)))

    def export_tilt(self, piece: int = 0) -> dict:
        """The tilted clocks' tables (of time piece ``piece``): lam, dl,
        inv_rate (float64), inv_rate32, dl32 (float32), still32 (int32, the
        row's threshold for the whole law)."""
        n = self.n
        out = dict(lam=np.zeros(n), dl=np.zeros(n), inv_rate=np.zeros(n),
                   inv_rate32=np.zeros(n, np.float32), dl32=np.zeros(n, np.float32),
                   still32=np.zeros(n, np.int32))
        keys = ["lam", "dl", "inv_rate", "inv_rate32", "dl32", "still32"]
        _check(self._lib.mlmc_export_tilt_piece(self._h, int(piece), *[_ptr(out[k]) for k in keys]))
        return out

    def export_proposal(self, piece: int = 0) -> dict:
        m = max(self.nnz, 1)
        out = dict(thr=np.zeros(m, np.uint32), keep_col=np.full(m, -1, np.int32),
                   keep_neg=np.zeros(m, np.uint8), alias_col=np.full(m, -1, np.int32),
                   alias_neg=np.zeros(m, np.uint8), lr_keep=np.zeros(m, np.float32),
                   lr_alias=np.zeros(m, np.float32))
        keys = ["thr", "keep_col", "keep_neg", "alias_col", "alias_neg", "lr_keep", "lr_alias"]
        _check(self._lib.mlmc_export_proposal_piece(self._h, int(piece),
                                                    *[_ptr(out[k]) for k in keys]))
        return out

    def info(self) -> dict:
        n, nnz, l0, t = ct.c_int64(), ct.c_int64(), ct.c_int32(), ct.c_double()
        _check(self._lib.mlmc_plan_info(self._h, ct.byref(n), ct.byref(nnz), ct.byref(l0),
                                        ct.byref(t)))
        return dict(n=n.value, nnz=nnz.value, l0=l0.value, t=t.value)

    def save_state(self) -> bytes:
        """The state of the last solve (row sums, totals and M_l per level,
        v, seed) as bytes, for mlmc_plan_load_state on a plan of the same
        matrix, t and schedule."""
        need = ct.c_size_t()
        _check(self._lib.mlmc_plan_save_state(self._h, None, 0, ct.byref(need)))
        buf = ct.create_string_buffer(need.value)
        _check(self._lib.mlmc_plan_save_state(self._h, buf, need.value, ct.byref(need)))
        return buf.raw[:need.value]

    def load_state(self, state: bytes):
        buf = ct.create_string_buffer(state, len(state))
        _check(self._lib.mlmc_plan_load_state(self._h, buf, len(state)))

    def expmv_resume(self, x, allow_not_converged: bool = False) -> int:
        """Continue the last (or loaded) mlmc_expmv with a fresh budget."""
        _need(x, 8 * self.n, "x")
        allow = (MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        return _check(self._lib.mlmc_expmv_resume(self._h, _ptr(x)), allow)

    def l2_window(self) -> dict:
        """The walk kernels' L2 access-policy window: bytes and hit ratio."""
        b, r = ct.c_int64(), ct.c_double()
        _check(self._lib.mlmc_plan_l2_window(self._h, ct.byref(b), ct.byref(r)))
        return dict(bytes=b.value, hit_ratio=r.value)

    def launch_count(self) -> int:
        return int(self._lib.mlmc_launch_count(self._h))


class Batch:
    """An mlmc_batch over plans (one problem per entry; repeat a plan for
    several right-hand sides)."""

    def __init__(self, plans, sched: Schedule = None, rel_tol: float = 1e-3, stream: int = 0):
        lib = load()
        self._lib = lib
        self._plans = list(plans)
        arr = (ct.c_void_p * len(self._plans))(*[p.handle for p in self._plans])
        self._h = ct.c_void_p()
        _check(lib.mlmc_batch_create(ct.byref(self._h), arr, len(self._plans),
                                     ct.byref(sched) if sched is not None else None,
                                     float(rel_tol), ct.c_void_p(stream)))

    def close(self):
        if self._h:
            self._lib.mlmc_batch_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def expmv(self, vs, xs, seeds, allow_not_converged: bool = False) -> int:
        k = len(self._plans)
        if len(vs) != k or len(xs) != k or len(seeds) != k:
            raise ValueError("one v, x and seed per problem")
        for p, v, x in zip(self._plans, vs, xs):
            _need(v, 8 * p.n, "v")
            _need(x, 8 * p.n, "x")
        va = (ct.c_void_p * k)(*[_ptr(v) for v in vs])
        xa = (ct.c_void_p * k)(*[_ptr(x) for x in xs])
        sa = (ct.c_uint64 * k)(*[int(s) for s in seeds])
        allow = (MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        return _check(self._lib.mlmc_batch_expmv(self._h, va, xa, sa), allow)

    def stats(self, problem: int):
        cap = 32
        arr = (LevelStats * cap)()
        nl = ct.c_int32()
        err = ct.c_double()
        _check(self._lib.mlmc_batch_stats(self._h, problem, arr, cap, ct.byref(nl), ct.byref(err)))
        levels = [{f: getattr(arr[j], f) for f, _ in LevelStats._fields_ if f != "pad"}
                  for j in range(nl.value)]
        return levels, err.value

    def info(self) -> dict:
        r, g, c = ct.c_int64(), ct.c_double(), ct.c_int32()
        _check(self._lib.mlmc_batch_info(self._h, ct.byref(r), ct.byref(g), ct.byref(c)))
        return dict(rounds=r.value, gpu_seconds=g.value, converged=c.value)

    def autotune(self):
        """Walks per lane for the three size buckets."""
        out = (ct.c_int32 * 4)()
        _check(self._lib.mlmc_batch_autotune(self._h, out, 4))
        return list(out)[:3]

    def block(self) -> int:
        """Threads per block of the round kernel chosen by the autotuner."""
        out = (ct.c_int32 * 4)()
        _check(self._lib.mlmc_batch_autotune(self._h, out, 4))
        return int(out[3])


class MLP:
    """The learned proposal's network (mlmc_mlp_*): 16 -> 64 -> 64 -> 1,
    BF16 tensor-core layers, FP32 master weights."""

    def __init__(self, seed: int = 1, stream: int = 0):
        lib = load()
        self._lib = lib
        self._h = ct.c_void_p()
        _check(lib.mlmc_mlp_create(ct.byref(self._h), ct.c_uint64(seed), ct.c_void_p(stream)))
        self.nparams = int(lib.mlmc_mlp_param_count())

    def close(self):
        if self._h:
            self._lib.mlmc_mlp_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    def params(self, set_to=None) -> np.ndarray:
        out = np.zeros(self.nparams, np.float32)
        if set_to is not None:
            _need(set_to, 4 * self.nparams, "params")
        _check(self._lib.mlmc_mlp_params(self._h, _ptr(set_to) if set_to is not None else None,
                                         _ptr(out)))
        return out

    def forward(self, x_bf16, n: int, z):
        _need(x_bf16, 2 * 16 * n, "x")
        _need(z, 4 * n, "z")
        _check(self._lib.mlmc_mlp_forward(self._h, _ptr(x_bf16), n, _ptr(z)))

    def loss_grad(self, x_bf16, y, n: int):
        _need(x_bf16, 2 * 16 * n, "x")
        _need(y, 4 * n, "y")
        loss = np.zeros(1, np.float32)
        grad = np.zeros(self.nparams, np.float32)
        _check(self._lib.mlmc_mlp_loss_grad(self._h, _ptr(x_bf16), _ptr(y), n, _ptr(loss),
                                            _ptr(grad)))
        return float(loss[0]), grad

    def train(self, x_bf16, y, n: int, steps: int, batch: int, lr: float, seed: int) -> float:
        loss = np.zeros(1, np.float32)
        _check(self._lib.mlmc_mlp_train(self._h, _ptr(x_bf16), _ptr(y), n, steps, batch,
                                        ct.c_float(lr), ct.c_uint64(seed), _ptr(loss)))
        return float(loss[0])

    def learn_proposal(self, plan, v, seed: int, pilot_walks: int = 256, steps: int = 300,
                       batch: int = 8192, lr: float = 3e-3, alpha: float = 0.1) -> float:
        _need(v, 8 * plan.n, "v")
        loss = np.zeros(1, np.float32)
        _check(self._lib.mlmc_learn_proposal(plan.handle, self._h, _ptr(v), ct.c_uint64(seed),
                                             pilot_walks, steps, batch, ct.c_float(lr),
                                             float(alpha), _ptr(loss)))
        return float(loss[0])

    def launch_count(self) -> int:
        return int(self._lib.mlmc_mlp_launch_count(self._h))

    def learn_tilt(self, plan, v, seed: int, pilot_walks: int = 256, steps: int = 300,
                   batch: int = 8192, lr: float = 3e-3, alpha: float = 0.1,
                   clocks: bool = True, rounds: int = 2, time_pieces: bool = False) -> float:
        """mlmc_learn_tilt: `rounds` pilot-train-install rounds of a proposal
        with tilted jumps and (clocks) holding times; with ``time_pieces``
        (and clocks) laws that change with time are candidates too.  Returns
        the last loss."""
        _need(v, 8 * plan.n, "v")
        loss = np.zeros(1, np.float32)
        tilt = TILT_JUMPS | (TILT_CLOCKS if clocks else 0)
        if time_pieces:
            if not clocks:
                raise ValueError("time pieces need tilted clocks")
            tilt |= TILT_TIME
        _check(self._lib.mlmc_learn_tilt(plan.handle, self._h, _ptr(v), ct.c_uint64(seed),
                                         pilot_walks, steps, batch, ct.c_float(lr), float(alpha),
                                         tilt, rounds, _ptr(loss)))
        return float(loss[0])
