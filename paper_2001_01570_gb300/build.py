"""Build libcgks.so (sm_103a) in-tree: paper_2001_01570_gb300/_build/libcgks.so,
and the diagnostics library libcgks_diag.so beside it (csrc/diag: checks of the
kernels' math routines against CUDA's and the FP64 throughput probe).

Each .cu translation unit is compiled by its own nvcc process (the tile-shape
instantiations of the stage kernel are the slow ones), then linked with
``nvcc -shared``.  CUDA runtime is linked statically so the libraries only
need the CUDA driver library (libcuda).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcgks.so")
DIAG_LIB = os.path.join(BUILD, "libcgks_diag.so")
# the same library compiled with CGKS_CHECK_BOUNDS: every kernel index checked against its buffer
# (a violation is recorded in the grid's status and the access skipped); for tests only
CHECK_BUILD = os.path.join(BUILD, "check")
CHECK_LIB = os.path.join(CHECK_BUILD, "libcgks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcgks")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _diag_sources():
    return sorted(glob.glob(os.path.join(CSRC, "diag", "*.cu")))


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(CSRC, "diag", "*.cu"))
                  + glob.glob(os.path.join(HERE, "..", "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(DIAG_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(DIAG_LIB))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build_check() -> str:
    """The bounds-checked build of libcgks (CHECK_LIB)."""
    if os.path.exists(CHECK_LIB) and all(os.path.getmtime(d) <= os.path.getmtime(CHECK_LIB) for d in _deps()):
        return CHECK_LIB
    return build(force=True, check_bounds=True)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, check_bounds: bool = False) -> str:
    if not force and not check_bounds and up_to_date():
        return LIB
    out_dir = CHECK_BUILD if check_bounds else BUILD
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources() + ([] if check_bounds else _diag_sources())
    objs = [os.path.join(out_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    ndiag = 0 if check_bounds else len(_diag_sources())
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DCGKS_CHECK_BOUNDS"] if check_bounds else [])

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose or ptxas_info:
        for l in logs:
            sys.stderr.write(l)
    targets = [(CHECK_LIB, objs)] if check_bounds else [(LIB, objs[:len(objs) - ndiag]),
                                                         (DIAG_LIB, objs[len(objs) - ndiag:])]
    for lib, parts in targets:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *parts]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return CHECK_LIB if check_bounds else LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
