"""The C-ABI library builds, loads and exports every function declared in include/*.h (CPU only)."""
import ctypes
import glob
import os
import re

from conftest import ROOT
from paper_2001_01570_gb300 import build as libbuild


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(?:cgks_status|const char\s*\*|long|int|void|double)\s+(cgks_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for n in ("cgks_create", "cgks_destroy", "cgks_set_state", "cgks_get_state", "cgks_step", "cgks_batch_step",
              "cgks_status_string", "cgks_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = libbuild.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(libbuild.build())
    lib.cgks_status_string.restype = ctypes.c_char_p
    assert lib.cgks_status_string(0) == b"ok"
    assert b"non-physical" in lib.cgks_status_string(5)


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """Every field of the binding's ctypes structs sits at the offset the C compiler gives it."""
    import shutil
    import subprocess

    import pytest

    from paper_2001_01570_gb300 import cgks

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"cgks_problem": cgks.cgks_problem, "cgks_serve_cfg": cgks.cgks_serve_cfg,
               "cgks_request": cgks.cgks_request}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cgks.h"', "int main(void) {"]
    for name, py in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, py in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(py), name
        for fname, _ in py._fields_:
            assert got[(name, fname)] == getattr(py, fname).offset, (name, fname)


def test_invalid_problems_are_rejected_before_any_device_work():
    """Argument checks of cgks_create run on the host: every one returns CGKS_E_INVAL with a
    message, on a machine with or without a GPU."""
    from paper_2001_01570_gb300 import cgks

    def bad(**kw):
        args = dict(dim=2, nx=8, ny=8, x0=0.0, x1=1.0)
        args.update(kw)
        p = cgks.make_problem(**args)
        for k, v in kw.items():
            if k in ("mu", "recon_vars", "order", "eps_tau", "weno_eps", "gamma", "cfl"):
                setattr(p, k, v)
        with __import__("pytest").raises(cgks.CgksError) as ei:
            cgks.cgks_create(p)
        assert ei.value.status == cgks.CGKS_E_INVAL
        assert lib.cgks_last_error()

    lib = cgks.load()
    lib.cgks_last_error.restype = ctypes.c_char_p
    bad(nx=0)
    bad(ny=0)
    bad(dim=3)
    bad(x1=0.0)
    bad(gamma=1.0)
    bad(cfl=0.0)
    bad(weno_eps=0.0)
    bad(mu=-1.0)
    bad(recon_vars=2)
    bad(order=7)
    bad(bc=(0, 1, 0, 0))                      # periodic on one x side only
    bad(bc=(1, 1, 0, 0), nx=1)                # a reflecting side needs two cells
    bad(bc=(2, 3, 0, 0), inflow=(0.0, 1.0, 0.0, 1.0))   # inflow density must be positive
