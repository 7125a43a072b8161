"""The stored oracle values under tests/golden/ (written by tests/golden/make_golden.py, which calls
only oracle/) are consistent with themselves and with the workloads they claim to hold: sample
indices inside the grid, sampled values bounded by the stored full-grid maxima, positive density,
the stated step counts; the one-file golden of the 256-grid batch holds whole size classes, and
where it samples a grid that also has a file of its own (an oracle run with another thread count),
both hold the same bits."""
import glob
import os

import numpy as np
import pytest

from conftest import GOLDEN
from paper_2001_01570_gb300 import workloads as wl

CASES = sorted(p for p in glob.glob(os.path.join(GOLDEN, "oracle_*.npz")) if "batched256" not in p)
BATCHED = os.path.join(GOLDEN, "oracle_batched256_100.npz")


@pytest.mark.parametrize("path", CASES, ids=[os.path.basename(p)[7:-4] for p in CASES])
def test_per_case_golden_is_consistent(path):
    g = np.load(path)
    idx, values, maxabs = g["idx"], g["values"], g["maxabs"]
    n = int(g["nx"]) * int(g["ny"])
    assert idx.ndim == 1 and np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < n
    assert values.shape == (12, idx.size) and maxabs.shape == (12,)
    assert np.all(np.abs(values) <= maxabs[:, None])
    assert np.all(values[0] > 0) and np.all(values[3] > 0)
    assert int(g["steps"]) > 0 and float(g["t"]) > 0 and float(g["last_dt"]) > 0
    if "floor" in g.files:
        assert np.all(g["floor"] >= 0) and np.all(g["floor"][:4] < 1e-8)


@pytest.fixture(scope="module")
def batched():
    if not os.path.exists(BATCHED):
        pytest.skip("oracle_batched256_100.npz not generated")
    return np.load(BATCHED)


def test_batched_golden_covers_whole_size_classes(batched):
    params = wl.batched_pulses()
    grids = [int(k) for k in batched["grid"]]
    assert len(set(grids)) == len(grids)
    nmax = max(params[k]["N"] for k in grids)
    assert set(grids) >= {k for k, p in enumerate(params) if p["N"] < nmax}
    assert np.all(batched["steps"] == 100)


def test_batched_golden_samples_are_consistent(batched):
    params = wl.batched_pulses()
    for j, k in enumerate(batched["grid"]):
        N = params[int(k)]["N"]
        idx, values, maxabs = batched["idx"][j], batched["values"][j], batched["maxabs"][j]
        assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < N * N
        assert np.all(np.abs(values) <= maxabs[:, None])
        assert np.all(values[0] > 0)
        assert 49.9 < float(batched["t"][j]) < 50.0        # 100 steps at CFL 0.5 of unit sound speed


def test_batched_golden_agrees_with_the_per_grid_files(batched):
    """Grids with a file of their own (1500 cells, an oracle run on all threads) and in the one-file
    golden (128 cells, one thread): the same final time, maxima and, on the cells both sample, values."""
    common = 0
    for j, k in enumerate(batched["grid"]):
        path = os.path.join(GOLDEN, f"oracle_pulse{int(k):03d}_100.npz")
        if not os.path.exists(path):
            continue
        g = np.load(path)
        assert float(g["t"]) == float(batched["t"][j])
        assert np.array_equal(g["maxabs"], batched["maxabs"][j])
        both, ia, ib = np.intersect1d(g["idx"], batched["idx"][j], return_indices=True)
        assert np.array_equal(g["values"][:, ia], batched["values"][j][:, ib])
        common += both.size
    if common == 0:
        pytest.skip("no grid sampled by both files yet")
