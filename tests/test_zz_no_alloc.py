"""The allocation-free entry point cgks_step_noalloc against the allocating path.

Callers that cannot let the library allocate device memory (own memory pools, fixed footprints,
regions where the allocator must not be re-entered) step a state they hold themselves through
cgks_step_noalloc, which keeps its scratch in fixed device arrays of the library.  Here the same
initial state is advanced by both entry points through the C ABI, over two consecutive calls
(3 steps, then 2 more), and the results must agree within the parity tolerance.  This file is
collected last on purpose."""
import numpy as np
import pytest

from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel_err(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    scale = np.abs(b).max(axis=1)
    diff = np.abs(a - b).max(axis=1)
    return np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), diff)


def test_noalloc_matches_allocating_path_on_two_calls():
    torch = pytest.importorskip("torch")
    spec, W = wl.shock_vortex(nx=72, ny=40, mach=1.2)
    prob = cgks.problem_from_spec(spec)
    # allocating path
    s = cgks.Solver(prob)
    s.set_state(W)
    s.step(3)
    ref1, t1, _ = s.get_state()
    s.step(2)
    ref2, t2, _ = s.get_state()
    s.close()
    # allocation-free path on a caller-owned device buffer
    planes = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    t = cgks.cgks_step_noalloc(prob, planes, 3, 0.0)
    torch.cuda.synchronize()
    out1 = planes.cpu().numpy()
    assert t == pytest.approx(t1, rel=1e-14)
    assert _rel_err(out1[:4], ref1[:4]).max() <= TOL
    assert _rel_err(out1[4:], ref1[4:]).max() <= 1e-9
    t = cgks.cgks_step_noalloc(prob, planes, 2, t)
    torch.cuda.synchronize()
    out2 = planes.cpu().numpy()
    assert t == pytest.approx(t2, rel=1e-14)
    assert _rel_err(out2[:4], ref2[:4]).max() <= TOL
    assert _rel_err(out2[4:], ref2[4:]).max() <= 1e-9


def test_noalloc_rejects_grids_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    prob = cgks.make_problem(2, 300, 300, 0.0, 1.0, 0.0, 1.0)
    planes = torch.zeros((12, 300, 300), dtype=torch.float64, device="cuda")
    with pytest.raises(cgks.CgksError) as ei:
        cgks.cgks_step_noalloc(prob, planes, 1, 0.0)
    assert ei.value.status == cgks.CGKS_E_INVAL
