"""GPU parity of the learned proposal's network (tcgen05 BF16 layers,
CUDA-core head, weight gradients and Adam) against the oracle's numpy MLP,
and the gain of the learned proposal over the plain jump law."""
import numpy as np
import pytest

import mlmc_inputs as I
from oracle import mlp as OM

from gpu_helpers import make_plan, stream_handle, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, OM.N_IN)) * 0.7
    x[:, 0] = 1.0
    y = np.sin(x[:, 1]) + 0.5 * x[:, 2] * x[:, 3] - 0.3 * x[:, 4]
    return x, y.astype(np.float32)


def _to_device_bf16(x):
    torch = torch_cuda()
    bits = OM.bf16_bits(x).astype(np.int16)
    return torch.from_numpy(bits.copy()).cuda()


@pytest.mark.parametrize("n", [128, 1000])
def test_forward_matches_oracle(n):
    torch = torch_cuda()
    from paper_1904_12754_gb300 import mlmc as M
    x, _ = _data(n, 1)
    with M.MLP(seed=3, stream=stream_handle()) as net:
        p = net.params()
        xd = _to_device_bf16(x)
        z = torch.zeros(n, dtype=torch.float32, device="cuda")
        net.forward(xd, n, z)
        torch.cuda.synchronize()
        z = z.cpu().numpy()
    zo, _, _ = OM.loss_and_grad(p.astype(np.float64), x, np.zeros(n))
    assert np.all(np.abs(z - zo) <= 2e-3 * (1.0 + np.abs(zo)))


def _gradient_bounds(p, x, y):
    """Per-element error bound of the GPU gradient against the oracle's.

    Every gradient entry is a sum over rows of products; the GPU forms them
    from BF16 operands with FP32 accumulation, the oracle in FP64 with the
    same BF16 rounding points.  Two effects separate them:
      - rounding: FP32 accumulation (relative 2^-24 per add, 2^-16 over a
        few hundred terms is generous) and a BF16 rounding of dA2 that can
        land on the other neighbour when the FP32 and FP64 values straddle a
        rounding boundary (relative 2^-8 on that term): bounded by
        2^-7 x (the same sum with every term in absolute value);
      - relu decisions: a pre-activation within rounding of 0 can take the
        other sign on the GPU, which moves that row's whole term: added in
        full for those rows (|a| below 1e-5 x the sum of |terms| of a).
    """
    q = OM.unpack(p.astype(np.float64))
    r = OM.round_bf16
    xb, W1, W2 = r(x), r(q["W1"]), r(q["W2"])
    a1 = xb @ W1 + q["b1"]
    s1 = np.abs(xb) @ np.abs(W1) + np.abs(q["b1"])
    h1 = r(np.maximum(a1, 0.0))
    a2 = h1 @ W2 + q["b2"]
    s2 = np.abs(h1) @ np.abs(W2) + np.abs(q["b2"])
    h2 = np.maximum(a2, 0.0)
    z = h2 @ q["w3"] + q["b3"][0]
    B = x.shape[0]
    dz = 2.0 * (z - y) / B
    u1 = np.abs(a1) <= 1e-5 * s1          # relu decisions that rounding can flip
    u2 = np.abs(a2) <= 1e-5 * s2
    m1, m2 = (a1 > 0) | u1, (a2 > 0) | u2  # every term that may be present
    da2a = np.abs(np.outer(dz, q["w3"])) * m2
    dh1a = np.abs(r(da2a)) @ np.abs(W2).T * 1.01
    da1a = dh1a * m1
    # rounding part (all terms in absolute value)
    absg = {"w3": np.abs(h2).T @ np.abs(dz), "b3": np.array([np.abs(dz).sum()]),
            "W2": np.abs(h1).T @ da2a, "b2": da2a.sum(axis=0),
            "W1": np.abs(xb).T @ da1a, "b1": da1a.sum(axis=0)}
    tol = {k: 2.0 ** -7 * v for k, v in absg.items()}
    # flip part: the full term of each row whose decision is uncertain
    flip2 = np.abs(np.outer(dz, q["w3"])) * u2
    tol["W2"] = tol["W2"] + np.abs(h1).T @ flip2
    tol["b2"] = tol["b2"] + flip2.sum(axis=0)
    flip1 = dh1a * u1
    tol["W1"] = tol["W1"] + np.abs(xb).T @ flip1
    tol["b1"] = tol["b1"] + flip1.sum(axis=0)
    return OM.pack(tol)


def test_gradients_match_oracle():
    # element by element: every one of the 5,441 parameters' gradient within
    # its own bound (rounding and relu decisions, _gradient_bounds) of the
    # oracle's; the bound is far below the gradient for nearly every entry
    torch = torch_cuda()
    from paper_1904_12754_gb300 import mlmc as M
    n = 777
    x, y = _data(n, 2)
    with M.MLP(seed=5, stream=stream_handle()) as net:
        p = net.params()
        loss, g = net.loss_grad(_to_device_bf16(x), torch.from_numpy(y).cuda(), n)
    _, lo, go = OM.loss_and_grad(p.astype(np.float64), x, y.astype(np.float64))
    assert abs(loss - lo) <= 1e-3 * abs(lo)
    tol = _gradient_bounds(p, x, y.astype(np.float64)) + 1e-7
    g = g.astype(np.float64)
    o = 0
    for name, shape in OM.SIZES:
        size = int(np.prod(shape))
        a, b, t = g[o:o + size], go[o:o + size], tol[o:o + size]
        bad = np.flatnonzero(np.abs(a - b) > t)
        assert bad.size == 0, (name, bad[:5], a[bad[:5]], b[bad[:5]], t[bad[:5]])
        o += size
    # the bound is informative: most entries are held to a small fraction of
    # their own magnitude
    big = np.abs(go) > 1e-4
    assert np.median(tol[big] / np.abs(go[big])) < 0.05


def test_training_reduces_loss():
    torch = torch_cuda()
    from paper_1904_12754_gb300 import mlmc as M
    n = 20000
    x, y = _data(n, 3)
    xd, yd = _to_device_bf16(x), torch.from_numpy(y).cuda()
    with M.MLP(seed=7, stream=stream_handle()) as net:
        l0, _ = net.loss_grad(xd, yd, n)
        net.train(xd, yd, n, steps=300, batch=2048, lr=3e-3, seed=1)
        l1, _ = net.loss_grad(xd, yd, n)
    assert l1 < 0.2 * l0


def test_learned_proposal_reduces_variance_and_stays_unbiased():
    # Barabasi-Albert n=3000, beta = 1/lambda_max: per-walk variance at l0
    # with the plain jump law and with the learned proposal, same walks count.
    torch = torch_cuda()
    from paper_1904_12754_gb300 import mlmc as M
    a = I.ba_graph(3000, 4, seed=11)
    t = 1.0 / I.lambda_max(a)
    v = np.ones(a.n)
    reps = 4096

    def level0(plan):
        dv = torch.from_numpy(v).cuda()
        s = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        tot = torch.zeros(8, dtype=torch.float64, device="cuda")
        plan.mlmcl(plan.info()["l0"], False, 1 << 20, reps, dv, 4242, s, tot)
        torch.cuda.synchronize()
        s, y2 = s.cpu().numpy(), float(tot[0])
        var = (y2 - (s * s).sum() / reps) / (reps - 1)
        return s / reps, var

    with make_plan(a, t, 1) as plan:
        m_plain, v_plain = level0(plan)
        with M.MLP(seed=9, stream=stream_handle()) as net:
            net.learn_proposal(plan, v, seed=77, pilot_walks=256, steps=300, batch=2048)
        m_learn, v_learn = level0(plan)
    assert v_learn < 0.9 * v_plain
    # both estimate the same per-row means: compare the totals within 4 sigma
    se = np.sqrt((v_plain + v_learn) / reps)
    assert abs(m_plain.sum() - m_learn.sum()) <= 4.0 * se


def test_learned_proposal_on_a_localized_right_hand_side():
    # 2D Laplacian, v a Gaussian bump: plain walks mostly end where v ~ 0;
    # the learned proposal steers jumps toward the bump.  Same walk count,
    # at least 3x smaller per-walk variance, and a mean within 4 sigma of
    # the FP64 judge.
    torch = torch_cuda()
    from oracle import reference as R
    from paper_1904_12754_gb300 import mlmc as M
    G = 48
    a = I.laplacian_2d(G)
    t = 2.0
    xs = np.arange(G) - (G - 1) / 2
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    v = np.exp(-(X ** 2 + Y ** 2) / 8.0).ravel()
    x = R.expmv(a.scipy(), t, v)
    reps = 2048

    def level0(plan):
        dv = torch.from_numpy(v).cuda()
        s = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        tot = torch.zeros(8, dtype=torch.float64, device="cuda")
        plan.mlmcl(plan.info()["l0"], False, 0, reps, dv, 31, s, tot)
        torch.cuda.synchronize()
        s, y2 = s.cpu().numpy(), float(tot[0])
        return s / reps, (y2 - (s * s).sum() / reps) / (reps - 1)

    with make_plan(a, t, 1) as plan:
        _, v_plain = level0(plan)
        with M.MLP(seed=2, stream=stream_handle()) as net:
            net.learn_proposal(plan, v, seed=5, pilot_walks=256, steps=300, batch=2048)
        m_learn, v_learn = level0(plan)
    assert v_learn < v_plain / 3.0
    # the level-l0 mean is the Strang approximation; compare the total to
    # exp(tA)v within the statistical error and the splitting error bound
    se = np.sqrt(v_learn / reps)
    assert abs(m_learn.sum() - x.sum()) <= 4.0 * se + 1e-2 * abs(x.sum())
