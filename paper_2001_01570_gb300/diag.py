"""Binding of libcgks_diag (csrc/diag/cgks_diag.cu): checks of the flux kernels' own math routines
against CUDA's, and the FP64 throughput of this GPU (the denominator of the kernels' roofline).

  python -m paper_2001_01570_gb300.diag      # prints the FP64 throughput table and the checks
"""
from __future__ import annotations

import ctypes
import json
import os

from . import build as _build

_lib = None

# operations of cgks_diag_fp64_rate, in its numbering
FP64_OPS = ("dfma, register operands", "dadd", "dmul", "dfma, immediate multiplicand",
            "add as fma(x, one, b)", "mul as fma(x, a, nzero)", "divide", "exp", "erfc", "rsqrt")


def load():
    global _lib
    if _lib is None:
        path = _build.DIAG_LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libcgks_diag is not built ({path} missing): run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        u64p = ctypes.POINTER(ctypes.c_ulonglong)
        L.cgks_diag_exp_neg_maxulp.argtypes = [ctypes.c_int, u64p]
        L.cgks_diag_rcp_maxulp.argtypes = [ctypes.c_int, u64p]
        L.cgks_diag_erfc_maxrel.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.cgks_diag_fp64_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what}: CUDA error {rc}")


def exp_neg_maxulp(n=1 << 24) -> int:
    v = ctypes.c_ulonglong()
    _ok(load().cgks_diag_exp_neg_maxulp(int(n), ctypes.byref(v)), "exp check")
    return int(v.value)


def rcp_maxulp(n=1 << 22) -> int:
    v = ctypes.c_ulonglong()
    _ok(load().cgks_diag_rcp_maxulp(int(n), ctypes.byref(v)), "rcp check")
    return int(v.value)


def erfc_maxrel(n=1 << 22) -> float:
    v = ctypes.c_double()
    _ok(load().cgks_diag_erfc_maxrel(int(n), ctypes.byref(v)), "erfc check")
    return float(v.value)


def fp64_rate(op=0, iters=4096) -> dict:
    """Throughput of one FP64 operation (index into FP64_OPS): G ops/s, per SM and cycle, SM MHz."""
    out = (ctypes.c_double * 3)()
    _ok(load().cgks_diag_fp64_rate(int(op), int(iters), out), "fp64 rate")
    return {"op": FP64_OPS[op], "gops": out[0], "per_sm_cycle": out[1], "sm_mhz": out[2]}


def main():
    _build.build()
    rows = []
    for op in range(len(FP64_OPS)):
        iters = 4096 if op < 6 else 512
        rows.append(fp64_rate(op, iters))
    for r in rows:
        print(f"{r['op']:32s} {r['gops']:10.2f} G/s  {r['per_sm_cycle']:6.3f} per SM and cycle  "
              f"SM clock {r['sm_mhz']:7.1f} MHz")
    checks = {"exp_neg_vs_exp_max_ulp": exp_neg_maxulp(), "rcp_vs_drcp_rn_max_ulp": rcp_maxulp(),
              "erfc_scaled_vs_erfc_max_rel": erfc_maxrel()}
    print(json.dumps(checks))


if __name__ == "__main__":
    main()
