"""Properties of the synthetic input generators."""
import numpy as np
import scipy.sparse as sp

import mlmc_inputs as I


def test_small_world_structure():
    n, k, p = 2000, 2, 0.1
    a = I.small_world(n, k, p, seed=3)
    m = a.scipy()
    assert (m != m.T).nnz == 0                      # symmetric
    assert m.diagonal().sum() == 0                  # no self-loops
    assert np.all(m.data == 1.0)                    # 0/1
    for d in range(1, k + 1):                       # every ring edge present
        i = np.arange(n)
        assert np.all(np.asarray(m[i, (i + d) % n]).ravel() == 1.0)
    deg = np.diff(a.row_ptr)
    assert deg.min() >= 2 * k
    # shortcuts: about p n k, each adds 2 to the degree sum (a few merge)
    extra = (deg.sum() - 2 * k * n) / 2
    assert abs(extra - p * n * k) < 5 * np.sqrt(p * n * k)
    assert np.array_equal(I.small_world(n, k, p, seed=3).col, a.col)   # seeded


def test_small_world_without_shortcuts_is_the_ring_lattice():
    a = I.small_world(50, 3, 0.0, seed=1)
    assert np.all(np.diff(a.row_ptr) == 6)
