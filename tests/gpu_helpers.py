"""Shared helpers of the GPU tests: problem set-up and oracle comparison."""
from __future__ import annotations

import numpy as np

import mlmc_inputs as I
from oracle import walker as W

EPS64 = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)


def torch_cuda():
    import torch
    return torch


def stream_handle() -> int:
    torch = torch_cuda()
    return torch.cuda.current_stream().cuda_stream


def make_plan(a, t, precision, l0=None, num_levels=3, max_levels=8, rel_tol=1e-2, pilot=64,
              max_jumps=1 << 20, stream=None, **kw):
    from paper_1904_12754_gb300 import mlmc as M
    sched = M.schedule_default(precision=precision, num_levels=num_levels, max_levels=max_levels,
                               pilot_walks=pilot, max_jumps_per_walk=max_jumps, **kw)
    if l0 is not None:
        sched.l0 = l0
    return M.Plan.from_csr(a, t, sched, rel_tol=rel_tol,
                           stream=stream if stream is not None else stream_handle())


def gpu_trace(plan, level, coarse, rep_begin, reps, v, seed):
    """All walks rep_begin..+reps of every row, recorded on the GPU."""
    from paper_1904_12754_gb300 import mlmc as M
    torch = torch_cuda()
    dv = torch.from_numpy(np.ascontiguousarray(v, np.float64)).cuda()
    rec = torch.zeros(plan.n * reps * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    plan.trace(level, coarse, rep_begin, reps, dv, seed, rec)
    torch.cuda.synchronize()
    return rec.cpu().numpy().view(M.WALK_RECORD_DTYPE)


def value_tolerance(orc, v, dl, level, fp64: bool):
    """Per-walk bound on |y_gpu - y_oracle|: relative part (1e-12 FP64 /
    1e-5 FP32) plus an absolute part covering rounding in the sums of
    +-dl/N terms that form the fine-minus-coarse exponent (they can cancel)."""
    n_grid = 2.0 ** level
    scale = np.abs(v[orc["end"]]) * np.exp(np.abs(orc["log_c"]) + np.abs(orc["log_f"]))
    terms = (orc["jumps"] + 3.0) * np.abs(dl).max() / n_grid
    if fp64:
        return 1e-12 * np.abs(orc["y"]) + 64 * EPS64 * scale * terms
    return 1e-5 * np.abs(orc["y"]) + 64 * EPS32 * scale * (terms + 1.0)


def compare_walks(got, orc, v, dl, level, fp64: bool, what: str = ""):
    """Index trajectories bit-exact, values within the stated tolerance."""
    assert got.shape == orc.shape
    for f in ("end", "jumps", "hash", "status"):
        bad = np.flatnonzero(got[f] != orc[f])
        assert bad.size == 0, f"{what}: {f} differs at {bad[:5]} ({got[f][bad[:5]]} vs {orc[f][bad[:5]]})"
    bad = np.flatnonzero(got["sign"] != orc["sign"])
    assert bad.size == 0, f"{what}: sign differs at {bad[:5]}"
    tol = value_tolerance(orc, v, dl, level, fp64)
    diff = np.abs(got["y"] - orc["y"])
    bad = np.flatnonzero(diff > tol)
    assert bad.size == 0, (f"{what}: y differs at {bad[:5]}: {got['y'][bad[:5]]} vs "
                           f"{orc['y'][bad[:5]]} (tol {tol[bad[:5]]})")


def oracle_walks(a, t, v, seed, fp64, rows, reps, level, coarse, tables=None, max_jumps=1 << 20):
    wk = W.Walker(a, t, v, seed=seed, precision=W.FP64 if fp64 else W.FP32, tables=tables,
                  max_jumps=max_jumps)
    return wk.walks(rows, reps, level, coarse), wk


def small_problems():
    """Matrices that span several work items, ragged sizes and the special
    rows: mixed signs, diagonal-only rows, stored zeros, a hub."""
    out = {}
    w = I.workload_c1()
    out["laplace2d_32"] = (w.a, w.t, w.v)
    a = I.random_sparse(301, 5, seed=17, signed=True, diag=True)
    out["signed_301"] = (a, 0.35, np.random.default_rng(3).standard_normal(a.n))
    b = I.ba_graph(3001, 4, seed=5)
    out["ba_3001"] = (b, 1.0 / I.lambda_max(b), np.ones(b.n))
    # hub + rows with only a diagonal + a row whose off-diagonals are stored zeros
    import scipy.sparse as sp
    rng = np.random.default_rng(8)
    n = 777
    r = np.concatenate([np.zeros(400, int), rng.integers(1, n, 900), np.arange(n)])
    c = np.concatenate([rng.choice(np.arange(1, n), 400, replace=False), rng.integers(0, n, 900),
                        np.arange(n)])
    vals = np.concatenate([rng.uniform(0.1, 2, 400) * rng.choice([-1, 1], 400),
                           rng.uniform(0.1, 1, 900) * rng.choice([-1, 1], 900),
                           rng.uniform(-1, 1, n)])
    m = sp.coo_matrix((vals, (r, c)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    hub = I.to_csr(m)
    # row 5: keep its entries but make the off-diagonals explicit zeros
    lo, hi = hub.row_ptr[5], hub.row_ptr[6]
    hub.val[lo:hi] = np.where(hub.col[lo:hi] == 5, hub.val[lo:hi], 0.0)
    out["hub_777"] = (hub, 0.2, rng.standard_normal(n))
    # rows whose stored lengths sit on both sides of the table builds'
    # block-per-row range [32, 8192]: 31, 32 (with its diagonal), 255, 256,
    # 8192, 8193 (with its diagonal); the other rows short
    n = 9000
    rows, cols, vals = [], [], []
    lengths = ((31, False), (32, True), (255, False), (256, True), (8192, False), (8193, True))
    for i, (length, diag) in enumerate(lengths):
        off = rng.choice(np.setdiff1d(np.arange(n), [i]), length - (1 if diag else 0),
                         replace=False)
        cc = np.sort(np.concatenate([off, [i]]) if diag else off)
        rows.append(np.full(cc.size, i))
        cols.append(cc)
        vals.append(rng.uniform(0.1, 1.0, cc.size) * rng.choice([-1, 1], cc.size) / length)
    for i in range(len(lengths), n):
        cc = np.unique(np.concatenate([rng.integers(0, n, 3), [i]]))
        rows.append(np.full(cc.size, i))
        cols.append(cc)
        vals.append(rng.uniform(-1, 1, cc.size))
    m = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    m.sort_indices()
    out["long_rows_9000"] = (I.to_csr(m), 0.3, rng.standard_normal(n))
    return out


def compare_fwd_walks(got, orc, fw, level, fp64, what):
    """Forward-mode walks: start, end, jumps, hash, status and sign bit for
    bit, values within the stated tolerance."""
    for f in ("pad", "end", "jumps", "hash", "status", "sign"):
        bad = np.flatnonzero(got[f] != orc[f])
        assert bad.size == 0, f"{what}: {f} differs at {bad[:5]} ({got[f][bad[:5]]} vs {orc[f][bad[:5]]})"
    # y = v_s (W/w_s) sign e^{...}: relative tolerance plus the rounding of
    # the +-dl/N sums that form the exponent (as for backward walks)
    s = orc["pad"]
    f = np.abs(fw.v[s]) * (fw.W / np.maximum(fw.w[s], 1))
    scale = f * np.exp(np.abs(orc["log_c"]) + np.abs(orc["log_f"]))
    terms = (orc["jumps"] + 3.0) * np.abs(fw.tables.dl).max() / 2.0 ** level
    if fp64:
        tol = 1e-12 * np.abs(orc["y"]) + 64 * EPS64 * scale * terms
    else:
        tol = 1e-5 * np.abs(orc["y"]) + 64 * EPS32 * scale * (terms + 1.0)
    bad = np.flatnonzero(np.abs(got["y"] - orc["y"]) > tol)
    assert bad.size == 0, f"{what}: y differs at {bad[:5]}: {got['y'][bad[:5]]} vs {orc['y'][bad[:5]]}"
