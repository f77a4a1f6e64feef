"""Algorithm 1 (the MLMC driver) on top of the oracle walker.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of Sec. 2.2 and Algorithm 1 (the GPU library's controller makes
the same ones):
  * the error target is eps = tol * ||x-hat||_2 (relative);
  * V_l is the total variance of one "sample" (one walk from every row):
    sum_i Var(Y_i), estimated unbiasedly as (sum Y^2 - sum_i S_i^2 / M)/(M-1);
  * C_l is the cost of one sample in events (jumps + 1 per walk);
  * M_l = ceil((2/eps^2) sqrt(V_l/C_l) sum_k sqrt(V_k C_k)) (Giles' optimum;
    Eq. 11 prints it garbled);
  * converged when sum_l V_l/M_l <= eps^2/2 and the bias estimate
    max(|m_L|, |m_{L-1}|/4)/3 <= eps/sqrt 2 (weak order 2, Eq. 13); otherwise
    L grows by one, up to the schedule's maximum.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import walker as W


@dataclass
class LevelState:
    level: int
    reps: int = 0
    sum_y: np.ndarray = None
    sum_y2: float = 0.0
    jumps: int = 0

    def mean(self) -> np.ndarray:
        return self.sum_y / max(self.reps, 1)

    def var_total(self) -> float:
        if self.reps < 2:
            return 0.0
        ss = float(np.dot(self.sum_y, self.sum_y))
        return max(0.0, (self.sum_y2 - ss / self.reps) / (self.reps - 1))


@dataclass
class Result:
    x: np.ndarray
    levels: list
    est_rel_err: float
    converged: bool
    events: int
    seconds: float
    info: dict = field(default_factory=dict)


def run(a, t: float, v: np.ndarray, tol: float, l0: int, num_levels: int, max_levels: int,
        pilot: int, seed: int, precision: int = W.FP64, max_reps: int = 1 << 40,
        time_budget: float = 1e30, nthreads: int = 0) -> Result:
    """Estimate exp(tA)v to relative RMS error ``tol`` (Algorithm 1)."""
    wk = W.Walker(a, t, v, seed, precision=precision)
    n = a.n
    t0 = time.perf_counter()
    levels = []

    def sample(st: LevelState, extra: int):
        coarse = st.level > l0
        s, s2, jmp, lim = wk.mlmcl(st.level, coarse, st.reps, extra, nthreads=nthreads)
        if lim:
            raise RuntimeError("oracle walk hit the jump limit")
        st.sum_y = s if st.sum_y is None else st.sum_y + s
        st.sum_y2 += s2
        st.jumps += jmp
        st.reps += extra

    for l in range(l0, l0 + num_levels):
        st = LevelState(l)
        sample(st, pilot)
        levels.append(st)
    converged = False
    while True:
        x = sum(st.mean() for st in levels)
        eps = tol * float(np.linalg.norm(x))
        vs = np.array([st.var_total() for st in levels])
        cs = np.array([n * (1.0 + st.jumps / (n * st.reps)) for st in levels])
        if eps > 0.0:
            total = float(np.sum(np.sqrt(vs * cs)))
            target = np.ceil(2.0 / eps ** 2 * np.sqrt(vs / cs) * total)
            for st, m in zip(levels, target):
                m = int(min(max(m, st.reps), max_reps))
                if m > st.reps:
                    sample(st, m - st.reps)
        x = sum(st.mean() for st in levels)
        eps = tol * float(np.linalg.norm(x))
        var = float(sum(st.var_total() / st.reps for st in levels))
        ml = float(np.linalg.norm(levels[-1].mean()))
        ml1 = float(np.linalg.norm(levels[-2].mean())) if len(levels) > 1 else ml
        bias = max(ml, ml1 / 4.0) / 3.0 if len(levels) > 1 else 0.0
        if var <= eps ** 2 / 2.0 * (1 + 1e-12) and bias <= eps / math.sqrt(2.0):
            converged = True
            break
        if time.perf_counter() - t0 > time_budget:
            break
        if bias > eps / math.sqrt(2.0) and len(levels) < max_levels:
            st = LevelState(levels[-1].level + 1)
            sample(st, pilot)
            levels.append(st)
            continue
        if all(st.reps >= max_reps for st in levels) or len(levels) >= max_levels and \
                bias > eps / math.sqrt(2.0):
            break
    x = sum(st.mean() for st in levels)
    nx = float(np.linalg.norm(x))
    var = float(sum(st.var_total() / st.reps for st in levels))
    est = math.sqrt(var) / nx if nx > 0 else 0.0
    events = int(sum(st.jumps + n * st.reps for st in levels))
    return Result(x, levels, est, converged, events, time.perf_counter() - t0)
