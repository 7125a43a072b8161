"""A battery of solves that exercises every indexing path of the kernels -- grids smaller than a
tile and than the stencil, every tile shape with ragged edges, every boundary type, 1D grids,
characteristic variables, the 6th-order variant, viscous flow, a batch mixing all of them, the
allocation-free entry point and the server -- run through whichever build of libcgks is loaded.
The test suite runs it on the bounds-checked build (CGKS_CHECK_BOUNDS: every kernel index checked
against its buffer) and compares with the normal build bit for bit.

  CGKS_LIBRARY=<build>/check/libcgks.so python -m paper_2001_01570_gb300.boundscheck out.npz
"""
from __future__ import annotations

import sys

import numpy as np

from . import cgks, workloads as wl


def _cases():
    out = []
    out.append(("shock-vortex 9x7", wl.shock_vortex(nx=9, ny=7, mach=1.2), 3, {}))
    out.append(("shock-vortex 2x3", wl.shock_vortex(nx=2, ny=3, mach=1.3), 3, {}))
    spec, W = wl.isentropic_vortex(6)
    out.append(("vortex 6x6", (spec, W), 3, {}))
    spec, W = wl.shock_vortex(nx=37, ny=23, mach=1.4)
    for shape in cgks.TILE_SHAPES:
        if shape != "64x1":
            out.append((f"shock-vortex 37x23 tiles {shape}", (spec, W), 2, {"tile": shape}))
    spec, W = wl.shock_vortex(nx=41, ny=19, mach=1.3)
    spec.recon_vars = 1
    out.append(("shock-vortex 41x19 characteristic", (spec, W), 3, {}))
    spec, W = wl.shock_vortex(nx=33, ny=21, mach=1.25)
    spec.order, spec.mu = 6, 1e-4
    out.append(("shock-vortex 33x21 6th order viscous", (spec, W), 3, {}))
    out.append(("shock reflection 30x8", wl.shock_reflection(30, 8), 3, {}))
    for n in (1, 3, 70):
        out.append((f"1D density wave {n}", wl.density_wave_1d(n, eps=0.2, cfl=0.3), 4, {}))
    out.append(("1D Sod 50", wl.shock_tube_1d(50), 4, {}))
    return out


def run_all():
    """{name: (planes, status)} of every case, plain path; then the 2D cases once more as one
    batch, through cgks_step_noalloc and through the server."""
    res = {}
    cases = _cases()
    for name, (spec, W), n, opt in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        if "tile" in opt:
            cgks.cgks_set_tile_shape(s.handle, opt["tile"])
        s.set_state(W)
        try:
            s.step(n)
            st = cgks.CGKS_OK
        except cgks.CgksError as e:
            st = e.status
        out = np.empty(s.shape)
        try:
            cgks.cgks_get_state(s.handle, out)
        except cgks.CgksError as e:
            st = st or e.status
        res[name] = (out, st)
        s.close()
    two_d = [(name, spec, W, n) for name, (spec, W), n, opt in cases if spec.dim == 2 and "tile" not in opt]
    solvers = []
    for name, spec, W, n in two_d:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        solvers.append(s)
    st = cgks.CGKS_OK
    try:
        cgks.cgks_batch_step([s.handle for s in solvers], 3)
    except cgks.CgksError as e:
        st = e.status
    for (name, spec, W, n), s in zip(two_d, solvers):
        out = np.empty(s.shape)
        try:
            cgks.cgks_get_state(s.handle, out)
            st2 = st
        except cgks.CgksError as e:
            st2 = st or e.status
        res["batched " + name] = (out, st2)
        s.close()
    try:
        import torch
        for name, spec, W, n in two_d:
            if spec.nx * spec.ny > cgks.NOALLOC_MAX_CELLS:
                continue
            planes = torch.from_numpy(np.ascontiguousarray(W)).cuda()
            try:
                cgks.cgks_step_noalloc(cgks.problem_from_spec(spec), planes, n, 0.0)
                st = cgks.CGKS_OK
            except cgks.CgksError as e:
                st = e.status
            torch.cuda.synchronize()
            res["noalloc " + name] = (planes.cpu().numpy(), st)
    except ImportError:
        pass
    srv = cgks.cgks_serve_start(hbm_budget_bytes=1e9, max_active=3, steps_per_round=2)
    try:
        ids = [cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, n) for name, spec, W, n in two_d]
        for rid, (name, spec, W, n) in zip(ids, two_d):
            out = np.empty_like(W)
            try:
                cgks.cgks_serve_wait(srv, rid, 300.0, out)
                st = cgks.CGKS_OK
            except cgks.CgksError as e:
                st = e.status
            res["served " + name] = (out, st)
    finally:
        cgks.cgks_serve_stop(srv)
    return res


def main():
    res = run_all()
    np.savez(sys.argv[1], names=np.array(list(res.keys())), status=np.array([v[1] for v in res.values()]),
             **{f"p{i}": v[0] for i, v in enumerate(res.values())})
    bad = [k for k, v in res.items() if v[1] != cgks.CGKS_OK]
    print(f"{len(res)} solves, {len(bad)} with a non-OK status: {bad}")


if __name__ == "__main__":
    main()
