"""The bounds-checked build of libcgks (CGKS_CHECK_BOUNDS: every index of a global record, state,
face-result or shared-memory access checked against its buffer; a violation is recorded in the
grid's status and reported as CGKS_E_CUDA) on a battery of solves that exercises every indexing
path (paper_2001_01570_gb300/boundscheck.py): no violation, and every result bit for bit the normal
build's.  The checked build runs in a child process (one CUDA library per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_2001_01570_gb300 import boundscheck, build, cgks

pytestmark = pytest.mark.gpu


def test_checked_build_finds_no_out_of_bounds_access_and_changes_no_result(tmp_path):
    lib = build.build_check()
    out = tmp_path / "checked.npz"
    env = dict(os.environ, CGKS_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "paper_2001_01570_gb300.boundscheck", str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    checked = np.load(out)
    names = list(checked["names"])
    status = dict(zip(names, checked["status"]))
    assert all(v == cgks.CGKS_OK for v in status.values()), {k: v for k, v in status.items() if v}
    normal = boundscheck.run_all()
    assert sorted(normal) == sorted(names)
    for i, name in enumerate(names):
        ref, st = normal[name]
        assert st == cgks.CGKS_OK, name
        assert np.array_equal(checked[f"p{i}"], ref), name
