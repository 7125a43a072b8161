"""The allocation-free entry point cgks_step_noalloc against the allocating path.

Callers that cannot let the library allocate device memory (own memory pools, fixed footprints,
regions where the allocator must not be re-entered) step a state they hold themselves through
cgks_step_noalloc, which keeps its scratch in fixed device arrays of the library.  Here the same
initial state is advanced by both entry points through the C ABI, over two consecutive calls
(3 steps, then 2 more).  The two paths run the same kernels on the same arithmetic and differ
only in where the scratch lives and in the tile decomposition (which never changes a result), so
they must agree bit for bit.  The cases cover the largest admissible grid (one side at
CGKS_NOALLOC_MAX_SIDE, CGKS_NOALLOC_MAX_CELLS cells), characteristic variables and the compact
6th-order variant.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu


def _cases():
    def big():
        spec, W = wl.shock_vortex(nx=cgks.NOALLOC_MAX_SIDE, ny=cgks.NOALLOC_MAX_CELLS // cgks.NOALLOC_MAX_SIDE,
                                  mach=1.2)
        return spec, W

    def char_vars():
        spec, W = wl.shock_vortex(nx=48, ny=26, mach=1.4)
        spec.recon_vars = 1
        return spec, W

    def sixth():
        spec, W = wl.isentropic_vortex(36)
        spec.order = 6
        return spec, W

    return [("shock-vortex 72x40", lambda: wl.shock_vortex(nx=72, ny=40, mach=1.2)),
            ("largest grid 4096x16", big), ("characteristic variables", char_vars),
            ("6th-order variant", sixth)]


@pytest.mark.parametrize("name,make", _cases(), ids=[c[0] for c in _cases()])
def test_noalloc_matches_allocating_path_on_two_calls(name, make):
    torch = pytest.importorskip("torch")
    spec, W = make()
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
    assert t == t1
    assert np.array_equal(out1, ref1)
    t = cgks.cgks_step_noalloc(prob, planes, 2, t)
    torch.cuda.synchronize()
    out2 = planes.cpu().numpy()
    assert t == t2
    assert np.array_equal(out2, ref2)


def test_noalloc_rejects_grids_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    prob = cgks.make_problem(2, 300, 300, 0.0, 1.0, 0.0, 1.0)
    planes = torch.zeros((12, 300, 300), dtype=torch.float64, device="cuda")
    with pytest.raises(cgks.CgksError) as ei:
        cgks.cgks_step_noalloc(prob, planes, 1, 0.0)
    assert ei.value.status == cgks.CGKS_E_INVAL
    side = cgks.NOALLOC_MAX_SIDE + 1
    prob = cgks.make_problem(2, side, 2, 0.0, 1.0, 0.0, 1.0)
    planes = torch.zeros((12, 2, side), dtype=torch.float64, device="cuda")
    with pytest.raises(cgks.CgksError) as ei:
        cgks.cgks_step_noalloc(prob, planes, 1, 0.0)
    assert ei.value.status == cgks.CGKS_E_INVAL
