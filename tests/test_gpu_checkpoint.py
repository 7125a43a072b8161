"""Checkpoint and resume through the C ABI: N steps, cgks_get_state (planes, t, step count),
cgks_restore_state into a new solver of the same problem, M more steps -- bit for bit the same as
N + M steps without interruption, with the same time and step count.  The time step of the first
resumed step is the CFL bound recomputed from the restored planes, so this also checks that the
bound of a restored state has the bits of the one the last step's update computed."""
import numpy as np
import pytest

from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu

N, M = 3, 4


def _cases():
    return [("shock-vortex 56x30, inflow/outflow/walls", lambda: wl.shock_vortex(nx=56, ny=30, mach=1.3)),
            ("vortex 40x40 periodic, characteristic variables", lambda: wl.isentropic_vortex(40)),
            ("1D Sod", lambda: wl.shock_tube_1d(90))]


@pytest.mark.parametrize("name,make", _cases(), ids=[c[0] for c in _cases()])
def test_plain_resume_is_bitwise(name, make):
    spec, W = make()
    if name.startswith("vortex"):
        spec.recon_vars = 1
    prob = cgks.problem_from_spec(spec)
    a = cgks.Solver(prob)
    a.set_state(W)
    a.step(N)
    ck, t_ck, steps_ck = a.get_state()
    assert steps_ck == N
    a.step(M)
    straight, t_straight, steps_straight = a.get_state()
    a.close()

    b = cgks.Solver(prob)
    b.restore(ck, t_ck, steps_ck)
    out0, t0, s0 = b.get_state()
    assert np.array_equal(out0, ck) and t0 == t_ck and s0 == N
    b.step(M)
    resumed, t_res, steps_res = b.get_state()
    b.close()
    assert steps_res == steps_straight == N + M
    assert t_res == t_straight
    assert np.array_equal(resumed, straight)


def test_batched_resume_is_bitwise():
    params = wl.batched_pulses(count=5, nmin=24, nmax=60)
    ics = [wl.acoustic_pulse(p["N"], p["A"], p["b"], p["cx"], p["cy"]) for p in params]
    ics.append(wl.shock_vortex(nx=44, ny=22, mach=1.45))

    def solvers():
        out = []
        for spec, W in ics:
            s = cgks.Solver(cgks.problem_from_spec(spec))
            s.set_state(W)
            out.append(s)
        return out

    first = solvers()
    cgks.cgks_batch_step([s.handle for s in first], N)
    cks = [s.get_state() for s in first]
    cgks.cgks_batch_step([s.handle for s in first], M)
    straight = [s.get_state() for s in first]
    for s in first:
        s.close()

    second = []
    for (spec, _), (planes, t, steps) in zip(ics, cks):
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.restore(planes, t, steps)
        second.append(s)
    cgks.cgks_batch_step([s.handle for s in second], M)
    for s, (ref, t_ref, steps_ref) in zip(second, straight):
        out, t, steps = s.get_state()
        assert steps == steps_ref == N + M
        assert t == t_ref
        assert np.array_equal(out, ref)
        s.close()


def test_restore_rejects_a_negative_step_count():
    spec, W = wl.isentropic_vortex(16)
    s = cgks.Solver(cgks.problem_from_spec(spec))
    with pytest.raises(cgks.CgksError) as ei:
        s.restore(W, 0.0, -1)
    assert ei.value.status == cgks.CGKS_E_INVAL
    s.close()
