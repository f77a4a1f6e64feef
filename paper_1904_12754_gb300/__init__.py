"""GB300-native multilevel Monte Carlo estimator of x = exp(tA)v.

The computation lives in ``libmlmc.so`` (CUDA, sm_103a; C ABI in
``include/mlmc.h``); :mod:`.mlmc` is a thin ctypes binding to it.
"""
from . import mlmc  # noqa: F401
from .mlmc import Plan, Schedule, schedule_default, MlmcError  # noqa: F401
