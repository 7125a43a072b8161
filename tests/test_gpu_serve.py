"""Continuous-batching server: requests of different sizes, kinds and step counts, submitted while
others run, with fewer slots than requests so that admission happens as slots free up; every
result must equal the same solve run alone (bit for bit: the batched launch performs the same
arithmetic per face and cell)."""
import threading
import time

import numpy as np
import pytest

from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu


def _alone(spec, W, nsteps):
    s = cgks.Solver(cgks.problem_from_spec(spec))
    s.set_state(W)
    s.step(nsteps)
    out, _, steps = s.get_state()
    s.close()
    assert steps == nsteps
    return out


def _cases():
    return [
        (wl.acoustic_pulse(40, 1e-3, 4.0, 10.0, 30.0), 9),
        (wl.isentropic_vortex(32), 5),
        (wl.shock_vortex(nx=48, ny=24, mach=1.3), 12),
        (wl.acoustic_pulse(64, 1e-5, 7.0, 50.0, 5.0), 3),
        (wl.isentropic_vortex(24), 7),
        (wl.shock_vortex(nx=40, ny=20, mach=1.05), 4),
    ]


def test_served_results_equal_alone_and_stats():
    cases = _cases()
    refs = [_alone(spec, W, n) for (spec, W), n in cases]
    srv = cgks.cgks_serve_start(hbm_budget_bytes=64e6, max_active=3, steps_per_round=2)
    ids = []
    try:
        def submitter():
            for (spec, W), n in cases:
                ids.append(cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, n))
                time.sleep(0.01)
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        outs = []
        for rid, ((spec, W), n) in zip(ids, cases):
            out = np.empty_like(W)
            cgks.cgks_serve_wait(srv, rid, 120.0, out)
            outs.append(out)
        stats = cgks.cgks_serve_stats(srv)
    finally:
        cgks.cgks_serve_stop(srv)
    for out, ref in zip(outs, refs):
        assert np.array_equal(out, ref)
    assert stats["completed"] == len(cases) and stats["failed"] == 0
    assert stats["p99_s"] >= stats["p50_s"] > 0.0
    assert stats["hbm_peak"] <= 64e6
    expected = sum(W.shape[1] * W.shape[2] * n for (spec, W), n in cases)
    assert stats["cell_updates"] == expected


def test_budget_limits_concurrency():
    """With a budget that holds one 64^2 solve at a time, requests run one after another."""
    spec, W = wl.acoustic_pulse(64, 1e-3, 5.0, 20.0, 20.0)
    one = cgks.cgks_problem_device_bytes(cgks.problem_from_spec(spec))
    assert one == 3 * 12 * 64 * 64 * 8 + 28 * 8 * (65 * 68 * 2) + 16 * 8 * (65 * 64 * 2) + 4096
    srv = cgks.cgks_serve_start(hbm_budget_bytes=one * 1.5, max_active=8, steps_per_round=1)
    try:
        ids = [cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, 3) for _ in range(3)]
        out = np.empty_like(W)
        for rid in ids:
            cgks.cgks_serve_wait(srv, rid, 120.0, out)
        stats = cgks.cgks_serve_stats(srv)
    finally:
        cgks.cgks_serve_stop(srv)
    assert stats["hbm_peak"] <= one * 1.5 and stats["completed"] == 3
    assert np.array_equal(out, _alone(spec, W, 3))


def test_composition_changes_keep_the_captured_graphs():
    """Twelve requests through four slots: the active set changes at almost every round, the queues
    are rewritten in place and no graph is captured beyond one per tuner candidate; the results
    equal the solves alone."""
    cases = [(wl.acoustic_pulse(24 + 4 * k, 1e-4, 3.0, 5.0 + k, 9.0), 3 + (k % 4)) for k in range(12)]
    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=4, steps_per_round=2)
    try:
        ids = [cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, n) for (spec, W), n in cases]
        outs = []
        for rid, ((spec, W), n) in zip(ids, cases):
            out = np.empty_like(W)
            cgks.cgks_serve_wait(srv, rid, 120.0, out)
            outs.append(out)
        stats = cgks.cgks_serve_stats(srv)
    finally:
        cgks.cgks_serve_stop(srv)
    assert stats["completed"] == 12
    assert 1 <= stats["graph_captures"] <= 6
    assert stats["gpu_s"] > 0.0
    for out, ((spec, W), n) in zip(outs, cases):
        assert np.array_equal(out, _alone(spec, W, n))


def test_server_and_batch_step_from_another_thread():
    """cgks_batch_step on one thread while the server runs requests on its own threads: both give
    the results of the solves alone."""
    serve_cases = [(wl.isentropic_vortex(40), 6), (wl.shock_vortex(nx=44, ny=22, mach=1.4), 5),
                   (wl.acoustic_pulse(48, 1e-5, 5.0, 12.0, 30.0), 7)]
    batch_cases = [wl.acoustic_pulse(36, 1e-3, 4.0, 9.0, 9.0), wl.isentropic_vortex(28)]
    batch_refs = [_alone(spec, W, 6) for spec, W in batch_cases]
    serve_refs = [_alone(spec, W, n) for (spec, W), n in serve_cases]
    errors = []

    def batch_thread():
        try:
            for _ in range(3):
                solvers = []
                for spec, W in batch_cases:
                    s = cgks.Solver(cgks.problem_from_spec(spec))
                    s.set_state(W)
                    solvers.append(s)
                cgks.cgks_batch_step([s.handle for s in solvers], 6)
                for s, ref in zip(solvers, batch_refs):
                    out, _, steps = s.get_state()
                    if steps != 6 or not np.array_equal(out, ref):
                        errors.append("batched result differs")
                    s.close()
        except Exception as e:  # noqa: BLE001
            errors.append(repr(e))

    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=2, steps_per_round=2)
    th = threading.Thread(target=batch_thread)
    try:
        th.start()
        for _ in range(2):
            ids = [cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, n) for (spec, W), n in serve_cases]
            for rid, ((spec, W), n), ref in zip(ids, serve_cases, serve_refs):
                out = np.empty_like(W)
                cgks.cgks_serve_wait(srv, rid, 120.0, out)
                assert np.array_equal(out, ref)
        th.join(timeout=300)
    finally:
        cgks.cgks_serve_stop(srv)
    assert not th.is_alive()
    assert not errors, errors


def test_nonphysical_request_fails_alone():
    """A request whose state turns non-physical (a cell with negative pressure) completes with
    CGKS_E_NONPHYSICAL and its last valid state, while the requests sharing its rounds finish with
    the results they have alone."""
    good = [(wl.isentropic_vortex(36), 6), (wl.acoustic_pulse(44, 1e-4, 4.0, 11.0, 30.0), 5)]
    spec_b, W_b = wl.acoustic_pulse(40, 1e-3, 4.0, 16.0, 16.0)
    bad = W_b.copy()
    bad[3, 5, 7] = 0.1 * bad[3, 5, 7] - 10.0
    refs = [_alone(spec, W, n) for (spec, W), n in good]
    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=3, steps_per_round=2)
    try:
        ids = [cgks.cgks_serve_submit(srv, cgks.problem_from_spec(good[0][0][0]), good[0][0][1], good[0][1]),
               cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec_b), bad, 4),
               cgks.cgks_serve_submit(srv, cgks.problem_from_spec(good[1][0][0]), good[1][0][1], good[1][1])]
        out_bad = np.empty_like(bad)
        with pytest.raises(cgks.CgksError) as ei:
            cgks.cgks_serve_wait(srv, ids[1], 120.0, out_bad)
        assert ei.value.status == cgks.CGKS_E_NONPHYSICAL
        for rid, ((spec, W), n), ref in zip((ids[0], ids[2]), good, refs):
            out = np.empty_like(W)
            cgks.cgks_serve_wait(srv, rid, 120.0, out)
            assert np.array_equal(out, ref)
        stats = cgks.cgks_serve_stats(srv)
    finally:
        cgks.cgks_serve_stop(srv)
    assert stats["completed"] == 2 and stats["failed"] == 1


def test_request_log(tmp_path):
    """With a log path the server appends one JSON line per finished request, with its grid, steps,
    status and the times of arrival, admission, first round and result (seconds since start)."""
    import json

    log = tmp_path / "serve.jsonl"
    cases = [(wl.isentropic_vortex(24), 4), (wl.acoustic_pulse(32, 1e-4, 3.0, 9.0, 20.0), 6),
             (wl.shock_vortex(nx=30, ny=16, mach=1.2), 3)]
    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=2, steps_per_round=2, log_path=log)
    try:
        ids = [cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, n) for (spec, W), n in cases]
        for rid, ((spec, W), n) in zip(ids, cases):
            cgks.cgks_serve_wait(srv, rid, 120.0, np.empty_like(W))
    finally:
        cgks.cgks_serve_stop(srv)
    lines = [json.loads(l) for l in log.read_text().splitlines()]
    assert sorted(l["id"] for l in lines) == sorted(ids)
    for l in lines:
        (spec, W), n = cases[ids.index(l["id"])]
        assert (l["nx"], l["ny"], l["steps"], l["status"]) == (spec.nx, spec.ny, n, cgks.CGKS_OK)
        assert 0.0 <= l["arrival_s"] <= l["admit_s"] <= l["first_round_s"] <= l["done_s"]
        assert l["latency_s"] == pytest.approx(l["done_s"] - l["arrival_s"], abs=1e-5)


@pytest.mark.parametrize("order", [cgks.CGKS_SERVE_LEAST_WORK_FIRST, cgks.CGKS_SERVE_ALL_ACTIVE])
def test_round_order(tmp_path, order):
    """Least remaining work first with a fill of 500 cells: the small solve (submitted first) runs
    alone, and the large one, admitted meanwhile, starts only after it; every solve in every round:
    both start together.  The results are the solves alone in both orders."""
    import json

    log = tmp_path / "order.jsonl"
    small, big = (wl.isentropic_vortex(24), 40), (wl.acoustic_pulse(96, 1e-4, 5.0, 40.0, 50.0), 40)
    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=4, steps_per_round=4, log_path=log, order=order,
                                fill_cells=500.0)
    try:
        ids = [cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, n) for (spec, W), n in (small, big)][::-1]
        outs = []
        for rid, ((spec, W), n) in zip(ids, (big, small)):
            out = np.empty_like(W)
            cgks.cgks_serve_wait(srv, rid, 120.0, out)
            outs.append(out)
    finally:
        cgks.cgks_serve_stop(srv)
    for out, ((spec, W), n) in zip(outs, (big, small)):
        assert np.array_equal(out, _alone(spec, W, n))
    rec = {l["id"]: l for l in map(json.loads, log.read_text().splitlines())}
    b, s = rec[ids[0]], rec[ids[1]]
    if order == cgks.CGKS_SERVE_LEAST_WORK_FIRST:
        assert b["first_round_s"] > s["first_round_s"] and s["done_s"] < b["done_s"]
    else:
        assert abs(b["first_round_s"] - s["first_round_s"]) < 0.05
