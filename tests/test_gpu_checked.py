"""The checked build (-DMLMC_CHECKED, compute-sanitizer being closed on this
pool): every table index a walk uses is compared with the table sizes before
it is used, and a walk that would leave them ends with a flag.  The parity
tests of the backward and forward walks run again, in a child process,
against the checked library: the same trajectories and values, and no flag
on valid tables."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_pass_on_the_checked_build():
    env = dict(os.environ, MLMC_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py", "tests/test_gpu_forward.py",
           "-k", "trajectories or tables or pilot"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout


def test_checked_library_is_the_one_loaded():
    env = dict(os.environ, MLMC_CHECKED="1")
    code = ("from paper_1904_12754_gb300 import mlmc as M; M.load(); "
            "print(M.library_path())")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().endswith("libmlmc_checked.so")
