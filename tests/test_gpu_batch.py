"""GPU parity of the controllers: single-plan mlmc_expmv and the batched
solver (mlmc_batch_*) against the CPU oracle.

With top-ups switched off (max_walks_per_row = pilot_walks) and every level
present from the start, an estimate is exactly the pilot sample
x = sum_l S_l / M of walks 0..M-1 of every level, which the oracle replays
walk by walk.  With top-ups on, the batch must reach its tolerance on every
problem against the FP64 judge."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import reference as R
from oracle import walker as W

from gpu_helpers import stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _pilot_only_schedule(precision, levels, pilot):
    from paper_1904_12754_gb300 import mlmc as M
    return M.schedule_default(precision=precision, num_levels=levels, max_levels=levels,
                              pilot_walks=pilot, max_walks_per_row=pilot)


def _oracle_pilot(a, t, v, seed, precision, l0, levels, pilot):
    wk = W.Walker(a, t, v, seed=seed, precision=W.FP64 if precision == 0 else W.FP32)
    x = np.zeros(a.n)
    for l in range(l0, l0 + levels):
        s, _, _, lim = wk.mlmcl(l, l > l0, 0, pilot)
        assert lim == 0
        x += s / pilot
    return x


def _problems():
    out = []
    a = I.random_sparse(257, 4, seed=41, signed=True, diag=True)
    out.append((a, 0.4, np.random.default_rng(1).standard_normal(a.n)))
    out.append((a, 0.4, np.random.default_rng(2).random(a.n)))   # second RHS, same plan
    b = I.laplacian_2d(19)
    out.append((b, 0.3, np.random.default_rng(3).random(b.n)))
    c = I.ba_graph(1500, 3, seed=9)
    out.append((c, 1.0 / np.diff(c.row_ptr).max(), np.ones(c.n)))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_expmv_pilot_sample_matches_oracle(precision):
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = _problems()[0]
    levels, pilot = 3, 96
    sched = _pilot_only_schedule(precision, levels, pilot)
    with M.Plan.from_csr(a, t, sched, rel_tol=1e-6, stream=stream_handle()) as plan:
        x = np.zeros(a.n)
        plan.expmv(v, x, seed=77, allow_not_converged=True)
        l0 = plan.info()["l0"]
    want = _oracle_pilot(a, t, v, 77, precision, l0, levels, pilot)
    tol = 1e-11 if precision == 0 else 2e-5
    assert np.abs(x - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_pilot_samples_match_oracle(precision):
    from paper_1904_12754_gb300 import mlmc as M
    probs = _problems()
    levels, pilot = 3, 64
    sched = _pilot_only_schedule(precision, levels, pilot)
    plans, cache = [], {}
    for a, t, _ in probs:
        key = (id(a), t)
        if key not in cache:
            cache[key] = M.Plan.from_csr(a, t, sched, rel_tol=1e-6, stream=stream_handle())
        plans.append(cache[key])
    seeds = [1001 + 17 * k for k in range(len(probs))]
    xs = [np.zeros(a.n) for a, _, _ in probs]
    with M.Batch(plans, sched, rel_tol=1e-6, stream=stream_handle()) as batch:
        batch.expmv([v for _, _, v in probs], xs, seeds, allow_not_converged=True)
        assert all(c in (4, 16, 64) for c in batch.autotune())
        assert batch.block() in (128, 256)
    tol = 1e-11 if precision == 0 else 2e-5
    for k, (a, t, v) in enumerate(probs):
        l0 = plans[k].info()["l0"]
        want = _oracle_pilot(a, t, v, seeds[k], precision, l0, levels, pilot)
        assert np.abs(xs[k] - want).max() <= tol * np.abs(want).max(), k
    for p in cache.values():
        p.close()


def test_batch_reaches_tolerance_on_every_problem():
    import torch
    from paper_1904_12754_gb300 import mlmc as M
    rng = np.random.default_rng(5)
    probs = []
    for k in range(12):
        g = int(rng.integers(8, 40))
        a = I.laplacian_2d(g) if k % 2 == 0 else I.laplacian_3d(max(3, g // 4))
        t = float(rng.uniform(0.1, 2.0))
        for r in range(1 + k % 3):
            probs.append((a, t, rng.random(a.n)))
    sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=3, max_levels=8,
                               pilot_walks=64, time_budget_s=120.0)
    tol = 1e-2
    plans, cache = [], {}
    for a, t, _ in probs:
        key = (id(a), t)
        if key not in cache:
            cache[key] = M.Plan.from_csr(a, t, sched, rel_tol=tol, stream=stream_handle())
        plans.append(cache[key])
    # device buffers for half of the problems, host for the rest
    vs = [torch.from_numpy(v).cuda() if k % 2 else v for k, (_, _, v) in enumerate(probs)]
    xs = [torch.zeros(a.n, dtype=torch.float64, device="cuda") if k % 2 else np.zeros(a.n)
          for k, (a, _, _) in enumerate(probs)]
    with M.Batch(plans, sched, rel_tol=tol, stream=stream_handle()) as batch:
        batch.expmv(vs, xs, [3 * k + 1 for k in range(len(probs))])
        info = batch.info()
        assert info["converged"] == len(probs)
        for k, (a, t, v) in enumerate(probs):
            x = xs[k].cpu().numpy() if k % 2 else xs[k]
            ref = R.expmv(a.scipy(), t, v)
            err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
            _, est = batch.stats(k)
            assert est <= tol
            assert err <= 2.5 * tol, (k, err)
    for p in cache.values():
        p.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_entry_pilot_sample_matches_oracle(precision):
    # Algorithm 2 for one entry: walks from row i only.
    from paper_1904_12754_gb300 import mlmc as M
    a, t, v = _problems()[0]
    levels, pilot = 3, 4096
    sched = _pilot_only_schedule(precision, levels, pilot)
    wk = W.Walker(a, t, v, seed=13, precision=W.FP64 if precision == 0 else W.FP32)
    with M.Plan.from_csr(a, t, sched, rel_tol=1e-9, stream=stream_handle()) as plan:
        l0 = plan.info()["l0"]
        for i in (0, 17, a.n - 1):
            xi = plan.expmv_entry(i, v, seed=13, allow_not_converged=True)
            want = 0.0
            for l in range(l0, l0 + levels):
                s, _, _, _ = wk.mlmcl(l, l > l0, 0, pilot, rows=(i, i + 1))
                want += s[i] / pilot
            tol = 1e-11 if precision == 0 else 2e-5
            assert abs(xi - want) <= tol * max(1.0, abs(want)), (i, xi, want)


def test_entry_and_total_communicability_reach_tolerance():
    from paper_1904_12754_gb300 import mlmc as M
    w = I.workload_c1()
    ref = R.expmv(w.a.scipy(), w.t, w.v)
    sched = M.schedule_default(precision=M.FP64, num_levels=3, max_levels=8)
    with M.Plan.from_csr(w.a, w.t, sched, rel_tol=1e-3, stream=stream_handle()) as plan:
        for i in (0, 500, 1023):
            xi = plan.expmv_entry(i, w.v, seed=3 + i)
            _, est = plan.stats()
            assert est <= 1e-3
            assert abs(xi - ref[i]) <= 4e-3 * abs(ref[i]), (i, xi, ref[i])
    b = I.ba_graph(3000, 4, seed=2)
    t = 1.0 / np.diff(b.row_ptr).max()
    tc_ref = R.expmv(b.scipy(), t, np.ones(b.n)).sum()
    sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=3, max_levels=8)
    with M.Plan.from_csr(b, t, sched, rel_tol=1e-4, stream=stream_handle()) as plan:
        tc = plan.expmv_sum(np.ones(b.n), seed=9)
        _, est = plan.stats()
    assert est <= 1e-4
    assert abs(tc - tc_ref) <= 4e-4 * tc_ref
