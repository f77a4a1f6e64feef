"""mlmc_trace_noalloc, the walk recorder that makes no device allocation,
against mlmc_trace through the C ABI.

Its scratch lives in static device memory shared by every call, so the
comparison is made on two calls in a row with different levels, replica
ranges and seeds: anything the first call leaves behind must not change the
second call's records.  A call is also captured into a CUDA graph in global
capture mode, which fails on any allocation, free or synchronisation, and
the graph's replay gives the same records; and an FP32 plan with a tilted
proposal records the same walks both ways.  Kept in its own file, collected
last."""
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


def test_noalloc_trace_is_captured_into_a_graph():
    # a cudaMalloc, cudaFree or stream synchronisation inside the call would
    # end the capture with an error
    import torch
    from gpu_helpers import make_plan
    from paper_1904_12754_gb300 import mlmc as M
    a = I.random_sparse(301, 5, seed=17, signed=True, diag=True)
    v = np.random.default_rng(3).standard_normal(a.n)
    side = torch.cuda.Stream()
    reps = 23
    with make_plan(a, 0.35, 1, stream=side.cuda_stream) as plan:
        dv = torch.from_numpy(v).cuda()
        want = _records(plan, "trace", 3, True, 7, reps, dv, 4321)
        rec = torch.zeros(plan.n * reps * M.WALK_RECORD_DTYPE.itemsize, dtype=torch.uint8,
                          device="cuda")
        plan.trace_noalloc(3, True, 7, reps, dv, 4321, rec)  # warm-up outside the capture
        torch.cuda.synchronize()
        rec.zero_()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            plan.trace_noalloc(3, True, 7, reps, dv, 4321, rec)
        graph.replay()
        torch.cuda.synchronize()
        got = rec.cpu().numpy().view(M.WALK_RECORD_DTYPE)
        for f in ("end", "jumps", "sign", "hash", "status"):
            assert np.array_equal(got[f], want[f]), f
        assert np.allclose(got["y"], want["y"], rtol=1e-5, atol=1e-30)


def test_noalloc_trace_with_a_tilted_proposal():
    import torch
    from gpu_helpers import make_plan
    b = I.ba_graph(1000, 4, seed=5)
    t = 1.0 / I.lambda_max(b)
    v = np.ones(b.n)
    h = np.exp(0.7 * np.random.default_rng(4).standard_normal(b.n)).astype(np.float32)
    with make_plan(b, t, 1) as plan:
        plan.set_tilt(h, 0.1, clocks=True)
        dv = torch.from_numpy(v).cuda()
        want = _records(plan, "trace", 2, True, 11, 31, dv, 77)
        got = _records(plan, "trace_noalloc", 2, True, 11, 31, dv, 77)
    for f in ("end", "jumps", "sign", "hash", "status"):
        assert np.array_equal(got[f], want[f]), f
    assert np.allclose(got["y"], want["y"], rtol=1e-5, atol=1e-30)
    assert want["jumps"].sum() > 0
