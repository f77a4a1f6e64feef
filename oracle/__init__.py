"""CPU oracle for the multilevel Monte Carlo estimator of x = exp(t A) v.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, FP64 judge of
the GPU library: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  It shares no code, headers,
tables or constant generators with the GPU path, and imports nothing from it.

Modules
  walker     ctypes binding to ``mlmc_oracle.c``: Philox4x32-10, neglog, the
             splitting of Sec. 2.1 (Eq. 1), Vose alias tables for the jump law
             of Eq. 12, and the walk of Algorithm 2 (MLMCL).
  reference  deterministic FP64 results: exp(tA) by Pade-13 scaling and
             squaring, exp(tA)v by truncated Taylor with scaling, the Strang
             products of Eq. 2 for every level, exact first and second moments
             of the level corrections, and brute-force path enumeration.
  mlmc       the driver of Algorithm 1 with Giles' optimal sample sizes
             (Eq. 11), running the oracle walker.
  mlp        numpy forward pass, loss and gradients of the proposal network
             with the GPU's BF16 rounding points, pinned by finite differences.

Every function whose result is not pinned by a test against something other
than itself says "parity unpinned" in its docstring.
"""
