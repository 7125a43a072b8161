"""Host-side logic of the server that needs no GPU: argument checks and budget rejection."""
import numpy as np
import pytest

from paper_2001_01570_gb300 import cgks, workloads as wl


def test_budget_rejection_and_bad_arguments():
    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e6, max_active=2, steps_per_round=2)
    try:
        spec, W = wl.acoustic_pulse(64, 1e-3, 4.0, 10.0, 10.0)     # 3 x 12 x 64^2 x 8 B > 1 MB
        with pytest.raises(cgks.CgksError) as ei:
            cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, 5)
        assert ei.value.status == cgks.CGKS_E_BUDGET
        p1 = cgks.make_problem(1, 10, 1, 0.0, 1.0)
        with pytest.raises(cgks.CgksError) as ei:
            cgks.cgks_serve_submit(srv, p1, np.zeros((6, 10)), 5)
        assert ei.value.status == cgks.CGKS_E_INVAL
        with pytest.raises(cgks.CgksError) as ei:
            cgks.cgks_serve_poll(srv, 12345)
        assert ei.value.status == cgks.CGKS_E_NOTFOUND
        st = cgks.cgks_serve_stats(srv)
        assert st["rejected"] == 1 and st["submitted"] == 0 and st["completed"] == 0
    finally:
        try:
            cgks.cgks_serve_stop(srv)
        except cgks.CgksError as e:    # without a GPU the scheduler could not start
            assert e.status == cgks.CGKS_E_CUDA


def test_bad_config():
    with pytest.raises(cgks.CgksError) as ei:
        cgks.cgks_serve_start(hbm_budget_bytes=0, max_active=2, steps_per_round=2)
    assert ei.value.status == cgks.CGKS_E_INVAL


def test_failed_scheduler_fails_requests_instead_of_hanging():
    """If the scheduler cannot run (here: no GPU, so it cannot create its streams), queued requests
    complete with its error and new submissions are refused with it, instead of waiting forever."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU (the scheduler must fail to start)")
    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=2, steps_per_round=2)
    try:
        spec, W = wl.acoustic_pulse(16, 1e-3, 3.0, 8.0, 8.0)
        prob = cgks.problem_from_spec(spec)
        statuses = []
        for _ in range(3):
            try:
                rid = cgks.cgks_serve_submit(srv, prob, W, 2)
            except cgks.CgksError as e:
                statuses.append(e.status)
                continue
            out = np.empty_like(W)
            try:
                cgks.cgks_serve_wait(srv, rid, 30.0, out)
                statuses.append(cgks.CGKS_OK)
            except cgks.CgksError as e:
                statuses.append(e.status)
        assert statuses and all(s == cgks.CGKS_E_CUDA for s in statuses), statuses
    finally:
        with pytest.raises(cgks.CgksError) as ei:
            cgks.cgks_serve_stop(srv)
        assert ei.value.status == cgks.CGKS_E_CUDA


def test_serve_config_checks():
    """An unknown round order, a non-positive fill for least-work-first rounds, a 1D tile shape and
    a request log that cannot be opened are rejected at start."""
    for kw in (dict(order=2), dict(order=cgks.CGKS_SERVE_LEAST_WORK_FIRST, fill_cells=0.0),
               dict(tile_shape=cgks.TILE_SHAPES.index("64x1")), dict(log_path="/nonexistent-dir/serve.log")):
        with pytest.raises(cgks.CgksError) as ei:
            cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=2, steps_per_round=2, **kw)
        assert ei.value.status == cgks.CGKS_E_INVAL
