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
