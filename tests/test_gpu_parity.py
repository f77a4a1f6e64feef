"""GPU parity: libmlmc (through the C ABI) against the CPU oracle.

Tables are compared bit for bit, walk trajectories bit for bit (end state,
jump count, sign, FNV hash of the visited states), walk values within 1e-12
(FP64 path) or 1e-5 (FP32 path) relative, per-row sums within rounding, and
level means within 4 standard errors of the exact moments."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W

from gpu_helpers import (compare_walks, gpu_trace, make_plan, oracle_walks, small_problems,
                         torch_cuda)

pytestmark = pytest.mark.gpu

PROBLEMS = small_problems()
PREC = {"fp64": 0, "fp32": 1}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _tables_equal(plan, a, t):
    got = plan.export_tables()
    tb = W.build_tables(a, t)
    nnz = a.nnz
    assert np.array_equal(got["deg"], tb.deg)
    for k in ("l_ii", "dl", "inv_rate"):
        ref = {"l_ii": tb.L, "dl": tb.dl, "inv_rate": tb.inv_rate}[k]
        assert np.array_equal(got[k].view(np.uint64), ref.view(np.uint64)), k
    assert np.array_equal(got["inv_rate32"].view(np.uint32), tb.inv_rate32.view(np.uint32))
    assert np.array_equal(got["dl32"].view(np.uint32), tb.dl32.view(np.uint32))
    mask = np.zeros(max(nnz, 1), bool)
    for i in range(a.n):
        mask[a.row_ptr[i]:a.row_ptr[i] + tb.deg[i]] = True
    for k in ("thr", "keep_col", "keep_neg", "alias_col", "alias_neg"):
        assert np.array_equal(got[k][mask], getattr(tb, k)[mask]), k
    return tb


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_tables_bit_exact(name):
    a, t, v = PROBLEMS[name]
    with make_plan(a, t, 0) as plan:
        _tables_equal(plan, a, t)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("level,coarse", [(2, False), (3, True), (7, True)])
def test_trajectories_bit_exact(name, prec, level, coarse):
    a, t, v = PROBLEMS[name]
    fp64 = prec == "fp64"
    reps = 37  # ragged: not a multiple of the warp width
    with make_plan(a, t, PREC[prec]) as plan:
        got = gpu_trace(plan, level, coarse, 5, reps, v, seed=1234)
    rows = np.repeat(np.arange(a.n), reps)
    rr = np.tile(np.arange(5, 5 + reps), a.n)
    orc, wk = oracle_walks(a, t, v, 1234, fp64, rows, rr, level, coarse)
    compare_walks(got, orc, v, wk.tables.dl, level, fp64, f"{name}/{prec}/l{level}")
    assert orc["jumps"].sum() > 0


@pytest.mark.parametrize("rep_begin", [(1 << 32) - 7, (1 << 40) + 3])
def test_high_replica_indices(rep_begin):
    # the counter's high replica bits (word 3, bits 8-31)
    a, t, v = PROBLEMS["signed_301"]
    with make_plan(a, t, 1) as plan:
        got = gpu_trace(plan, 3, True, rep_begin, 16, v, seed=77)
    orc, wk = oracle_walks(a, t, v, 77, False, np.repeat(np.arange(a.n), 16),
                           np.tile(np.arange(rep_begin, rep_begin + 16), a.n), 3, True)
    compare_walks(got, orc, v, wk.tables.dl, 3, False, "high reps")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mlmcl_row_sums_match_oracle(prec):
    torch = torch_cuda()
    a, t, v = PROBLEMS["signed_301"]
    fp64 = prec == "fp64"
    reps = 200
    with make_plan(a, t, PREC[prec]) as plan:
        dv = torch.from_numpy(v).cuda()
        s = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        tot = torch.zeros(8, dtype=torch.float64, device="cuda")
        plan.mlmcl(4, True, 0, reps, dv, 9, s, tot)
        torch.cuda.synchronize()
        s, tot = s.cpu().numpy(), tot.cpu().numpy()
    wk = W.Walker(a, t, v, seed=9, precision=W.FP64 if fp64 else W.FP32)
    os_, oy2, oj, ol = wk.mlmcl(4, True, 0, reps)
    scale = np.abs(os_).max()
    assert np.abs(s - os_).max() <= (1e-11 if fp64 else 1e-4) * scale
    assert abs(tot[0] - oy2) <= (1e-11 if fp64 else 1e-4) * oy2
    assert tot[1] == oj and tot[2] == a.n * reps and tot[3] == ol == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("level,coarse", [(1, False), (3, True)])
def test_level_means_within_4_sigma_of_exact(prec, level, coarse):
    torch = torch_cuda()
    a = I.random_sparse(7, 3, seed=31, signed=True, diag=True)
    t = 0.8
    v = np.random.default_rng(2).random(7) - 0.4
    m1, m2 = R.level_moments(a.dense(), t, v, level, coarse)
    reps = 1 << 18
    with make_plan(a, t, PREC[prec]) as plan:
        dv = torch.from_numpy(v).cuda()
        s = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        tot = torch.zeros(8, dtype=torch.float64, device="cuda")
        plan.mlmcl(level, coarse, 0, reps, dv, 2024, s, tot)
        torch.cuda.synchronize()
        s = s.cpu().numpy()
    var = m2 - m1 * m1
    noisy = var > 1e-12 * np.maximum(m2, 1e-300)
    z = (s[noisy] / reps - m1[noisy]) / np.sqrt(var[noisy] / reps)
    assert np.abs(z).max() <= 4.0
    # rows without jumps are deterministic: exact up to rounding
    fixed = ~noisy
    assert np.all(np.abs(s[fixed] / reps - m1[fixed]) <= 1e-6 * np.abs(m1[fixed]) + 1e-300)


def test_expmv_c1_reaches_tolerance_fp64():
    w = I.workload_c1()
    ref = R.expmv(w.a.scipy(), w.t, w.v)
    with make_plan(w.a, w.t, 0, num_levels=w.num_levels, rel_tol=w.tol) as plan:
        x = np.zeros(w.a.n)
        plan.expmv(w.v, x, seed=11)
        levels, est = plan.stats()
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    assert est <= w.tol
    assert err <= 2.0 * w.tol
    assert levels[0]["level"] == 2  # Eq. 16 for this matrix
    # Lemma 2: V_l falls about 4x per level above l0
    vs = [lv["var"] for lv in levels[1:]]
    assert all(vs[k + 1] < vs[k] / 2 for k in range(len(vs) - 1))


def test_expmv_device_and_host_buffers_agree():
    torch = torch_cuda()
    a, t, v = PROBLEMS["ba_3001"]
    with make_plan(a, t, 1, rel_tol=1e-2) as plan:
        xh = np.zeros(a.n)
        plan.expmv(v, xh, seed=5)
        dv = torch.from_numpy(v).cuda()
        xd = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        plan.expmv(dv, xd, seed=5)
        torch.cuda.synchronize()
    assert np.array_equal(xh, xd.cpu().numpy()) or \
        np.abs(xh - xd.cpu().numpy()).max() <= 1e-12 * np.abs(xh).max()


def test_diagonal_matrix_is_exact():
    import scipy.sparse as sp
    d = np.linspace(-2, 1, 50)
    a = I.to_csr(sp.diags(d))
    v = np.random.default_rng(1).random(50)
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-6)):
        with make_plan(a, 0.7, PREC[prec], rel_tol=1e-3) as plan:
            x = np.zeros(50)
            plan.expmv(v, x, seed=1)
            _, est = plan.stats()
        # no variance: the estimate is zero up to the rounding of the sums
        assert est <= 1e-7
        assert np.abs(x - np.exp(0.7 * d) * v).max() <= tol * np.abs(x).max()


def test_time_zero_returns_v():
    a, _, v = PROBLEMS["signed_301"]
    with make_plan(a, 0.0, 0) as plan:
        x = np.zeros(a.n)
        plan.expmv(v, x, seed=1)
    assert np.array_equal(x, v)


def test_stochastic_generator_gives_ones_exactly():
    import scipy.sparse as sp
    a0 = I.random_sparse(500, 4, seed=6, signed=False, diag=False).scipy()
    q = I.to_csr(a0 - sp.diags(np.asarray(a0.sum(axis=1)).ravel()))
    for prec in (0, 1):
        with make_plan(q, 1.5, prec, rel_tol=1e-3) as plan:
            x = np.zeros(500)
            plan.expmv(np.ones(500), x, seed=4)
        # d_i = a_ii + L_ii is zero up to the rounding of the two row sums
        assert np.abs(x - 1.0).max() <= 1e-12


def test_single_row_matrix():
    a = I.CSR(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([-0.5]))
    with make_plan(a, 2.0, 0) as plan:
        x = np.zeros(1)
        plan.expmv(np.array([3.0]), x, seed=1)
    assert abs(x[0] - 3.0 * np.exp(-1.0)) <= 1e-14


@pytest.mark.parametrize("bad", ["unsorted", "col_range", "nan", "row_ptr"])
def test_invalid_csr_is_rejected(bad):
    from paper_1904_12754_gb300 import mlmc as M
    a = I.random_sparse(20, 3, seed=1)
    rp, col, val = a.row_ptr.copy(), a.col.copy(), a.val.copy()
    if bad == "unsorted":
        i = int(np.argmax(np.diff(rp) >= 2))
        col[rp[i]], col[rp[i] + 1] = col[rp[i] + 1], col[rp[i]]
    elif bad == "col_range":
        col[3] = 20
    elif bad == "nan":
        val[4] = np.nan
    else:
        rp[5] = rp[4] - 1
    with pytest.raises(M.MlmcError) as e:
        M.Plan(20, rp, col, val, 1.0, M.schedule_default())
    assert e.value.status == M.MLMC_ERR_INVALID_ARG


def test_walk_limit_is_an_error_not_a_hang():
    from paper_1904_12754_gb300 import mlmc as M
    a = I.ring_graph(64)
    with make_plan(a, 20.0, 1, max_jumps=3, l0=0) as plan:
        got = gpu_trace(plan, 2, False, 0, 4, np.ones(64), seed=3)
        orc, _ = oracle_walks(a, 20.0, np.ones(64), 3, False, np.repeat(np.arange(64), 4),
                              np.tile(np.arange(4), 64), 2, False, max_jumps=3)
        assert np.array_equal(got["status"], orc["status"]) and got["status"].max() == 1
        with pytest.raises(M.MlmcError) as e:
            plan.expmv(np.ones(64), np.zeros(64), seed=1)
        assert e.value.status == M.MLMC_ERR_WALK_LIMIT
