"""The host operation count of the kernels' formulas (paper_2001_01570_gb300/opcount.py), which
gives the roofline's algorithmic FP64 count in the convention add/sub/mul 1, fma 2, divide,
square root, reciprocal, exponential, erfc 1 each.  Pinned against hand counts of the update
formulas (Sec. 2.2, Eq. step-hyper-1; Sec. 3.1, Eq. compact-deriv-1; the CFL bound of Sec. 4) and
checked for the special functions a smooth inviscid flux evaluation calls."""
import pytest

from paper_2001_01570_gb300 import opcount, workloads as wl


@pytest.fixture(scope="module")
def vortex64():
    spec, W = wl.isentropic_vortex(64)
    return spec, opcount.count_step(spec, W)


def test_update_counts_match_the_formulas(vortex64):
    spec, res = vortex64
    # stage 1, per variable: W* and R (3 subtractions, 2 multiplications each) and the four
    # gradient differences (1 subtraction, 1 multiplication each): 20
    assert res["update1"]["flop_per_cell"] == 4 * 20
    # stage 2, per variable: W^{n+1} (3 sub, 2 mul) and two gradient increments (sub, mul, add);
    # CFL bound: 1/rho, U, V, the kinetic energy (2 mul, add, mul), gamma-1, E-KE, p, c (2 mul, sqrt),
    # 2 nu (2 mul), both directions' signal speed (add, mul, add) and dx / speed
    assert res["update2"]["flop_per_cell"] == 4 * 12 + 23


def test_flux_special_functions_per_segment(vortex64):
    spec, res = vortex64
    n = spec.nx
    segments = 2 * n * n + 2 * n            # every face once (periodic: the last faces too)
    c = res["flux1"]["counts"]
    # per Gauss point: the two half-line moment sets (one exp and one erfc each), two 1/sqrt(2 theta),
    # reciprocals of the three densities and of p_l + p_r; per segment also one reciprocal per
    # variable for the WENO-Z weights along the face and one for the two slopes: 16
    # (the collision-time exponential is skipped where dt > 80 tau, as for eps_tau = 0.01)
    assert c["exp"] == 4 * segments and c["erfc"] == 4 * segments
    assert c["sqrt"] == 4 * segments
    assert c["rcp"] == 16 * segments
    assert c["div"] == 0
    # the record kernel: one reciprocal per (face row, variable) with WENO-Z
    assert res["records1"]["counts"]["exp"] == 0 and res["records1"]["counts"]["rcp"] > 0


def test_bench_constants_are_the_count_on_the_bench_grid():
    """bench.py's per-cell formula counts for the 2048^2 vortex follow from the per-unit counts
    (record item with and without the WENO-Z pair, face segment, cell) measured on 64^2 and 128^2:
    the smooth vortex takes no data-dependent branch, so each unit's count is the same on every
    grid."""
    import importlib.util
    import os

    import numpy as np
    from conftest import ROOT

    spec_b = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec_b)
    spec_b.loader.exec_module(bench)
    per = {}
    for n in (64, 128):
        spec, W = wl.isentropic_vortex(n)
        per[n] = opcount.count_step(spec, W)

    def units(n):
        inner, outer = 2 * (n + 1) * (n + 2), 2 * (n + 1) * 2     # record rows with / without WENO-Z
        return 4 * inner, 4 * outer, 2 * n * n + 2 * n, n * n      # record items, segments, cells

    # records: two unknown per-item counts from two grids
    A = np.array([units(n)[:2] for n in (64, 128)], dtype=float)
    b = np.array([per[n]["records1"]["flop"] for n in (64, 128)], dtype=float)
    item_in, item_out = np.linalg.solve(A, b)
    n = 2048
    ii, io, seg, cells = units(n)
    assert (item_in * ii + item_out * io) / cells == pytest.approx(bench.OPCOUNT_FLOP_PER_CELL["records"], rel=2e-6)
    for stage in (1, 2):
        per_seg = per[128][f"flux{stage}"]["flop"] / units(128)[2]
        assert per[64][f"flux{stage}"]["flop"] / units(64)[2] == pytest.approx(per_seg, rel=1e-12)
        assert per_seg * seg / cells == pytest.approx(bench.OPCOUNT_FLOP_PER_CELL["flux"][stage], rel=2e-6)
        assert per[128][f"update{stage}"]["flop_per_cell"] == bench.OPCOUNT_FLOP_PER_CELL["update"][stage]
