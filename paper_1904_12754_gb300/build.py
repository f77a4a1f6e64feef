"""Build libmlmc.so (CUDA, sm_103a) in-tree with nvcc.

Each translation unit is compiled in parallel, then linked into
``paper_1904_12754_gb300/_build/libmlmc.so``.  Only one architecture is
generated: ``-gencode arch=compute_103a,code=sm_103a``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmlmc.so")
# The checked build (-DMLMC_CHECKED: every table index a walk uses is
# compared with the table sizes; see the walk kernels) in its own folder.
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libmlmc_checked.so")
SOURCES = ["mlmc_abi.cu", "mlmc_tables.cu", "mlmc_walk.cu", "mlmc_reduce.cu", "mlmc_noalloc.cu",
           "mlmc_batch.cu", "mlmc_mlp.cu",
           "mlmc_forward.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmlmc")


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "mlmc.h"))
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(verbose: bool = False, force: bool = False, extra_flags=None,
          checked: bool = False) -> str:
    """Compile (if needed) and return the path of libmlmc.so (or, with
    checked=True, of the checked build libmlmc_checked.so)."""
    out_dir, lib_path = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = FLAGS + (["-DMLMC_CHECKED"] if checked else []) + list(extra_flags or [])
    jobs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        if force or _stale(obj, path):
            jobs.append([nvcc, *ARCH, *flags, "-c", path, "-o", obj])
    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return r
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(out_dir, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or not os.path.exists(lib_path):
        tmp = lib_path + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
