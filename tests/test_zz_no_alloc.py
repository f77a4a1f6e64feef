"""mlmc_trace_noalloc, the walk recorder that makes no device allocation,
against mlmc_trace through the C ABI.

Its scratch lives in static device memory shared by every call, so the
comparison is made on two calls in a row with different levels, replica
ranges and seeds: anything the first call leaves behind must not change the
second call's records.  Kept in its own file, collected last."""
import numpy as np
import pytest

import mlmc_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _records(plan, which, level, coarse, rep_begin, reps, dv, seed):
    import torch
    from paper_1904_12754_gb300 import mlmc as M
    rec = torch.zeros(plan.n * reps * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    getattr(plan, which)(level, coarse, rep_begin, reps, dv, seed, rec)
    torch.cuda.synchronize()
    return rec.cpu().numpy().view(M.WALK_RECORD_DTYPE)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_trace_matches_trace_on_two_calls(precision):
    import torch
    from gpu_helpers import make_plan
    a = I.random_sparse(301, 5, seed=17, signed=True, diag=True)
    v = np.random.default_rng(3).standard_normal(a.n)
    rtol = 1e-12 if precision == 0 else 1e-5
    with make_plan(a, 0.35, precision) as plan:
        dv = torch.from_numpy(v).cuda()
        calls = [(3, True, 5, 37, 1234), (2, False, (1 << 32) - 3, 19, 99)]
        for level, coarse, rep_begin, reps, seed in calls:
            want = _records(plan, "trace", level, coarse, rep_begin, reps, dv, seed)
            got = _records(plan, "trace_noalloc", level, coarse, rep_begin, reps, dv, seed)
            for f in ("end", "jumps", "sign", "hash", "status"):
                assert np.array_equal(got[f], want[f]), f
            assert np.all(np.abs(got["y"] - want["y"]) <= rtol * np.abs(want["y"]) + 1e-300)
            assert want["jumps"].sum() > 0


def test_noalloc_trace_rejects_more_rows_than_its_scratch():
    import scipy.sparse as sp
    import torch
    from gpu_helpers import make_plan
    from paper_1904_12754_gb300 import mlmc as M
    n = (1 << 18) + 1
    a = I.to_csr(sp.diags(np.full(n, -0.5)))
    with make_plan(a, 1.0, 1) as plan:
        dv = torch.ones(n, dtype=torch.float64, device="cuda")
        rec = torch.zeros(n * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        with pytest.raises(M.MlmcError) as e:
            plan.trace_noalloc(0, False, 0, 1, dv, 1, rec)
        assert e.value.status == M.MLMC_ERR_INVALID_ARG
        assert "262144" in str(e.value)
