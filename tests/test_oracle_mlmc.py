"""The oracle's Algorithm 1 driver reaches its tolerance against the FP64
judge (C1: 2D Laplacian 32x32, FP64 walks, rel. RMS 1e-2)."""
import numpy as np

import mlmc_inputs as I
from oracle import mlmc as M
from oracle import reference as R
from oracle import walker as W


def test_oracle_mlmc_reaches_tolerance_on_laplacian():
    w = I.workload_c1()
    ref = R.expmv(w.a.scipy(), w.t, w.v)
    tb = W.build_tables(w.a, w.t)
    l0 = R.choose_l0(tb.dl / w.t, tb.L, w.t)
    # Eq. 16 with d_max = max(|d_i|, L_ii) = 4/h^2 and t = h^2/2: log2(4) = 2
    assert l0 == 2
    res = M.run(w.a, w.t, w.v, w.tol, l0=l0, num_levels=w.num_levels, max_levels=8,
                pilot=64, seed=5)
    assert res.converged
    err = np.linalg.norm(res.x - ref) / np.linalg.norm(ref)
    # the controller aims at RMS error tol; allow 2x for one draw of the noise
    assert err <= 2.0 * w.tol
    assert res.est_rel_err <= w.tol
