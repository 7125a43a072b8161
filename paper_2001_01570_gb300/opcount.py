"""Host count of the FP64 operations of one time step of the CUDA kernels' own formulas
(libcgks_opcount, csrc/opcount/cgks_opcount.cpp), in the convention of the roofline's algorithmic
count: add, subtract, multiply 1; fused multiply-add 2; divide, square root, reciprocal,
exponential, erfc 1 each (however the GPU expands them).

  python -m paper_2001_01570_gb300.opcount [N]     # the isentropic vortex on N x N (default 256)
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import sys

import numpy as np

from . import cgks

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "opcount", "cgks_opcount.cpp")
LIB = os.path.join(HERE, "_build", "libcgks_opcount.so")
KINDS = ("add", "mul", "fma", "div", "sqrt", "rcp", "exp", "erfc")
LAUNCHES = ("records1", "flux1", "update1", "records2", "flux2", "update2")
_lib = None


def _deps():
    d = os.path.join(HERE, "csrc")
    return [SRC] + [os.path.join(d, f) for f in os.listdir(d) if f.endswith((".cuh", ".h"))]


def build(force=False) -> str:
    """g++ the host counter (it includes the kernels' device headers)."""
    if not force and os.path.exists(LIB) and all(os.path.getmtime(p) <= os.path.getmtime(LIB) for p in _deps()):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++20", "-fPIC", "-shared", "-Wno-unknown-pragmas",
                    "-I", cuda_inc,
                    "-o", tmp, SRC], check=True)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.cgks_opcount_step.argtypes = [ctypes.POINTER(cgks.cgks_problem), ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_ulonglong)]
        L.cgks_opcount_step.restype = ctypes.c_int
        L.cgks_host_step.argtypes = [ctypes.POINTER(cgks.cgks_problem), ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p]
        L.cgks_host_step.restype = ctypes.c_int
        _lib = L
    return _lib


def flops(counts: dict) -> float:
    """Operations in the roofline convention (FMA = 2, every other operation 1)."""
    return sum(v * (2 if k == "fma" else 1) for k, v in counts.items())


def count_step(spec, W) -> dict:
    """Per launch: the operation counts of one step of the kernels on this grid, and per cell."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = (ctypes.c_ulonglong * (6 * len(KINDS)))()
    rc = load().cgks_opcount_step(ctypes.byref(cgks.problem_from_spec(spec)), W.ctypes.data, out)
    if rc != 0:
        raise RuntimeError(f"cgks_opcount_step returned {rc}")
    cells = spec.nx * spec.ny
    res = {}
    for i, name in enumerate(LAUNCHES):
        c = {k: int(out[i * len(KINDS) + j]) for j, k in enumerate(KINDS)}
        res[name] = {"counts": c, "flop": flops(c), "flop_per_cell": flops(c) / cells}
    return res


def host_step(spec, W, fused: bool) -> np.ndarray:
    """One step of the kernels' arithmetic on the host (dt from the CFL bound of W): the
    three-kernel arrangement, or the fused one (cgks_fused.cuh).  2D."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.empty_like(W)
    rc = load().cgks_host_step(ctypes.byref(cgks.problem_from_spec(spec)), W.ctypes.data, int(bool(fused)),
                               out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"cgks_host_step returned {rc}")
    return out


def main():
    from . import workloads as wl
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 256
    spec, W = wl.isentropic_vortex(n)
    res = count_step(spec, W)
    print(json.dumps({"grid": f"isentropic vortex {n}x{n}", "per_cell": {k: v["flop_per_cell"] for k, v in res.items()},
                      "counts": {k: v["counts"] for k, v in res.items()}}, indent=1))


if __name__ == "__main__":
    main()
