"""Write the oracle's expected values for the full-size parity tests.

Calls only oracle/ (and the shared input generators).  For each case the oracle runs the stated
number of steps on the full grid; stored are: the final time and step count, the per-plane maximum
|value| over the whole grid (the normalisation of the relative error), and all 12 planes at a
seeded sample of cells.

  python tests/golden/make_golden.py vortex512     # isentropic vortex 512^2, 200 steps
  python tests/golden/make_golden.py shockvortex   # shock-vortex 1024x512, 400 steps
  python tests/golden/make_golden.py pulses        # 8 smallest grids of the 256-grid batch, 100 steps
  python tests/golden/make_golden.py pulses16      # 16 grids of the batch across its size quantiles
                                                   # (smallest to largest, 65^2..501^2), 100 steps
  python tests/golden/make_golden.py served        # 20 sampled requests of the served stream at
                                                   # their stated N and step count (every kind; shock-
                                                   # vortex from Mach 1.07 to 1.50), with the oracle's
                                                   # own rounding floor (y-mirrored run)
  python tests/golden/make_golden.py batched256 [workers]
                                                   # every grid of the 256-grid batch, 100 steps, smallest
                                                   # first, 128 cells each, into one file that is rewritten
                                                   # after each grid (a rerun skips the grids it holds)
  python tests/golden/make_golden.py vortex2048    # isentropic vortex 2048^2 (the bench grid), 2 steps
  python tests/golden/make_golden.py vortex2048o6  # the same grid, compact 6th-order variant, 1 step
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2001_01570_gb300 import workloads as wl  # noqa: E402

NSAMPLE = 1500

# the stratified sample of the 256 batched grids: sorted by N, 16 evenly spaced ranks
def pulse_quantile_grids(params, count=16):
    order = sorted(range(len(params)), key=lambda k: params[k]["N"])
    ranks = np.linspace(0, len(params) - 1, count).round().astype(int)
    return [order[r] for r in ranks]


# requests of the served stream (seed 2001) that the oracle runs at their stated size and step
# count: the cheapest of each kind plus weak pulses and the strongest shocks
SERVED_SAMPLE = (1661, 1283, 1920, 1208, 10, 1356, 1919, 221,
                 1126, 432, 1679, 205, 565, 1250, 669, 646, 1732, 1063, 776, 1014)


def sample_cells(ny, nx, seed):
    rng = np.random.default_rng(seed)
    n = min(NSAMPLE, nx * ny)
    flat = rng.choice(nx * ny, size=n, replace=False)
    return np.sort(flat)


def mirror_y(W):
    """The state mirrored in y (rows reversed): the y-momentum, its x-gradient and the y-gradients
    of the other variables change sign."""
    W = W[:, ::-1, :].copy()
    for p in (2, 6, 8, 9, 11):
        W[p] *= -1.0
    return W


def write_case(name, spec, W, nsteps, seed, floor=False):
    """The oracle's result after nsteps steps at NSAMPLE seeded cells.  floor=True also stores the
    oracle's own rounding floor for this run: the oracle on the y-mirrored problem, mirrored back,
    against the oracle (the same arithmetic on the same values, rounded in another order), per
    plane relative to the plane's maximum."""
    t0 = time.time()
    P = O.make_problem(**spec.as_kwargs())
    Wn, t, steps, last_dt = O.run(P, W, nsteps)
    idx = sample_cells(spec.ny, spec.nx, seed)
    planes = Wn.reshape(Wn.shape[0], -1)
    maxabs = np.abs(planes).max(axis=1)
    extra = {}
    if floor:
        Wm = mirror_y(O.run(P, mirror_y(W), nsteps)[0]).reshape(Wn.shape[0], -1)
        extra["floor"] = np.abs(Wm - planes).max(axis=1) / np.where(maxabs > 0, maxabs, 1.0)
    np.savez_compressed(os.path.join(HERE, f"oracle_{name}.npz"), idx=idx, values=planes[:, idx],
                        maxabs=maxabs, t=t, steps=steps, last_dt=last_dt, nx=spec.nx, ny=spec.ny, **extra)
    msg = "" if not floor else "; rounding floor " + " ".join(f"{x:.1e}" for x in extra["floor"][:4])
    print(f"{name}: {steps} steps to t={t:.6f} in {time.time() - t0:.0f} s{msg}", flush=True)


BATCHED_FILE = os.path.join(HERE, "oracle_batched256_100.npz")
BATCHED_NSAMPLE = 128


def _batched_grid(k):
    """One grid of the batch on one oracle thread: its sampled cells after 100 steps."""
    p = wl.batched_pulses()[k]
    spec, W = wl.acoustic_pulse(p["N"], p["A"], p["b"], p["cx"], p["cy"])
    Wn, t, steps, _ = O.run(O.make_problem(**spec.as_kwargs()), W, 100, threads=1)
    rng = np.random.default_rng(25600 + k)
    idx = np.sort(rng.choice(spec.nx * spec.ny, size=BATCHED_NSAMPLE, replace=False))
    planes = Wn.reshape(Wn.shape[0], -1)
    return k, idx, planes[:, idx], np.abs(planes).max(axis=1), t, steps


def batched256(workers):
    import multiprocessing as mp
    params = wl.batched_pulses()
    done = {}
    if os.path.exists(BATCHED_FILE):
        g = np.load(BATCHED_FILE)
        for j, k in enumerate(g["grid"]):
            done[int(k)] = (g["idx"][j], g["values"][j], g["maxabs"][j], float(g["t"][j]), int(g["steps"][j]))
    todo = [k for k in sorted(range(len(params)), key=lambda k: (params[k]["N"], k)) if k not in done]
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers) as pool:
        for k, idx, values, maxabs, t, steps in pool.imap(_batched_grid, todo):
            done[k] = (idx, values, maxabs, t, steps)
            ks = sorted(done)
            tmp = BATCHED_FILE + ".tmp.npz"
            np.savez_compressed(tmp, grid=np.array(ks), idx=np.stack([done[j][0] for j in ks]),
                                values=np.stack([done[j][1] for j in ks]),
                                maxabs=np.stack([done[j][2] for j in ks]),
                                t=np.array([done[j][3] for j in ks]), steps=np.array([done[j][4] for j in ks]))
            os.replace(tmp, BATCHED_FILE)
            print(f"grid {k} ({params[k]['N']}^2): {steps} steps to t={t:.6f}; {len(done)} of {len(params)} "
                  f"grids after {time.time() - t0:.0f} s", flush=True)


def main(which):
    if which == "vortex512":
        spec, W = wl.isentropic_vortex(512)
        write_case("vortex512_200", spec, W, 200, seed=512)
    elif which == "shockvortex":
        spec, W = wl.shock_vortex(1024, 512)
        write_case("shockvortex1024x512_400", spec, W, 400, seed=1024)
    elif which == "vortex2048":
        spec, W = wl.isentropic_vortex(2048)
        write_case("vortex2048_2", spec, W, 2, seed=2048)
    elif which == "vortex2048o6":
        spec, W = wl.isentropic_vortex(2048)
        spec.order = 6
        write_case("vortex2048o6_1", spec, W, 1, seed=2049)
    elif which == "pulses":
        params = wl.batched_pulses()
        order = sorted(range(len(params)), key=lambda k: params[k]["N"])[:8]
        for k in order:
            p = params[k]
            spec, W = wl.acoustic_pulse(p["N"], p["A"], p["b"], p["cx"], p["cy"])
            write_case(f"pulse{k:03d}_100", spec, W, 100, seed=k)
    elif which == "pulses16":
        params = wl.batched_pulses()
        for k in pulse_quantile_grids(params):
            p = params[k]
            if os.path.exists(os.path.join(HERE, f"oracle_pulse{k:03d}_100.npz")):
                continue
            spec, W = wl.acoustic_pulse(p["N"], p["A"], p["b"], p["cx"], p["cy"])
            write_case(f"pulse{k:03d}_100", spec, W, 100, seed=k)
    elif which == "batched256":
        batched256(int(sys.argv[2]) if len(sys.argv) > 2 else max(1, (os.cpu_count() or 2) - 1))
    elif which == "served":
        reqs = {r["id"]: r for r in wl.served_requests()}
        for rid in SERVED_SAMPLE:
            r = reqs[rid]
            if os.path.exists(os.path.join(HERE, f"oracle_request{rid:04d}_{r['steps']}.npz")):
                continue
            spec, W = wl.request_problem(r)
            write_case(f"request{rid:04d}_{r['steps']}", spec, W, r["steps"], seed=20010 + rid, floor=True)
        # the Mach 1.48 request before its vortex reaches the shock (the rounding floor of the
        # full run is set by that interaction)
        if not os.path.exists(os.path.join(HERE, "oracle_request1919_150.npz")):
            spec, W = wl.request_problem(reqs[1919])
            write_case("request1919_150", spec, W, 150, seed=21919, floor=True)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1])
