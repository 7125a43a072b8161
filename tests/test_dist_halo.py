"""The domain decomposition that a single large grid would use across GPUs, on CPU ranks (gloo,
world size 2) with the oracle: the grid is split in x, each rank steps its half with the
neighbour's two boundary columns (all 12 planes) received before each stage and the time step
reduced to the minimum over ranks; the result equals the undivided grid bit for bit.  (Every run
of this library uses one GPU; this pins the exchange pattern the decomposition needs.)"""
import multiprocessing as mp
import os
import socket

import numpy as np
import torch.multiprocessing as tmp

from conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem_parts():
    import oracle as O
    from paper_2001_01570_gb300 import workloads as wl
    spec, W = wl.shock_vortex(nx=48, ny=24, mach=1.3)      # inflow / outflow in x, reflecting in y
    kw = spec.as_kwargs()
    return O, kw, W


def _worker(rank, world, port, nsteps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        O, kw, W = _problem_parts()
        nx = kw["nx"]
        half = nx // world
        lo, hi = rank * half, (rank + 1) * half
        bc = list(kw["bc"])
        if rank > 0:
            bc[0] = O.BC_HALO
        if rank < world - 1:
            bc[1] = O.BC_HALO
        kwr = dict(kw, nx=half, bc=tuple(bc))
        P = O.make_problem(**kwr)
        Wr = np.ascontiguousarray(W[:, :, lo:hi])
        ny = kw["ny"]

        def exchange(stage, state, halo):
            # boundary columns of every rank: [first two, last two] (12 planes x ny each)
            mine = torch.from_numpy(np.concatenate([state[:, :, :2], state[:, :, -2:]], axis=2).copy())
            allc = [torch.empty_like(mine) for _ in range(world)]
            dist.all_gather(allc, mine)
            if rank > 0:                              # low side: the left rank's last columns
                left = allc[rank - 1].numpy()
                halo[0, :, 0, :] = left[:, :, 3]      # ghost column -1
                halo[0, :, 1, :] = left[:, :, 2]      # ghost column -2
            if rank < world - 1:                      # high side: the right rank's first columns
                right = allc[rank + 1].numpy()
                halo[1, :, 0, :] = right[:, :, 0]     # ghost column nx
                halo[1, :, 1, :] = right[:, :, 1]     # ghost column nx + 1

        for _ in range(nsteps):
            dt = torch.tensor([O.cfl_dt(P, Wr)], dtype=torch.float64)
            dist.all_reduce(dt, op=dist.ReduceOp.MIN)
            Wr = O.step2d_halo(P, Wr, float(dt[0]), exchange)
        out[rank] = Wr.tobytes()
        out["shape%d" % rank] = Wr.shape
    finally:
        dist.destroy_process_group()


def test_two_rank_x_split_equals_the_whole_grid():
    import sys
    sys.path.insert(0, ROOT)
    O, kw, W = _problem_parts()
    nsteps = 4
    ref, _, steps, _ = O.run(O.make_problem(**kw), W, nsteps)
    assert steps == nsteps
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), nsteps, out), nprocs=world, join=True)
    parts = [np.frombuffer(out[r], dtype=np.float64).reshape(out["shape%d" % r]) for r in range(world)]
    got = np.concatenate(parts, axis=2)
    assert np.array_equal(got, ref)
