"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake (a wrong coefficient, sign or index, a dropped term, a transposed
operand) in a copy of the oracle's C source, builds that copy with the oracle's own flags, and runs
the pin tests named beside it against the planted library (``CGKS_ORACLE_LIB``): at least one of
them must fail.  A control run of every named pin against an unplanted copy, through the same
override, must pass, so a failure comes from the planted mistake and not from the harness.

Everything here is CPU-only and touches only the oracle; the CUDA library is not involved.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle as O

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

R = "tests/test_oracle_recon.py::"
K = "tests/test_oracle_kinetic.py::"
S = "tests/test_oracle_scheme.py::"
V = "tests/test_oracle_viscous.py::"
C = "tests/test_oracle_characteristic.py::"
T = "tests/test_oracle_tangential.py::"
X = "tests/test_oracle_sixth_order.py::"

# (what the mistake is, text in the oracle source, its replacement, pins expected to catch it)
MUTANTS = [
    ("P7 value: one coefficient of Eq. (recons-8th-val)", "185.0 * Q[2]", "158.0 * Q[2]",
     [R + "test_linear_recon_exact_up_to_degree_7"]),
    ("P7 slope: one sign", "- 99.0 * hQp[2]", "+ 99.0 * hQp[2]",
     [R + "test_linear_recon_exact_up_to_degree_7"]),
    ("P7 second derivative: a dropped term", "- hQp[0] - 9.0 * hQp[1]", "- 9.0 * hQp[1]",
     [R + "test_linear_recon_exact_up_to_degree_7"]),
    ("candidate slope at the interface: the power factor dropped",
     "sl += m * c[m] * ipow(0.5, m - 1)", "sl += c[m] * ipow(0.5, m - 1)",
     [R + "test_indicators_slopes_match_symbolic_definition"]),
    ("smoothness indicator: wrong integral of xi^e", "ipow(-0.5, e + 1)) / (e + 1)",
     "ipow(-0.5, e + 1)) / (e + 2)", [R + "test_indicators_slopes_match_symbolic_definition"]),
    ("beta_1 not taken from the cubic on the reduced stencil",
     "beta[1] = poly_beta(POLY_DEFS[7].deg, c);", "(void)c;",
     [R + "test_indicators_slopes_match_symbolic_definition"]),
    ("global reference Z: wrong indicator index", "3.0 * (beta[0] - beta[4])", "3.0 * (beta[0] - beta[3])",
     [X + "test_weno6_smooth_order", S + "test_shock_tube_vs_exact_riemann"]),
    ("WENO-Z weight: the 1 dropped", "dlin[k] * (1.0 + Z / (beta[k] + eps))", "dlin[k] * (Z / (beta[k] + eps))",
     [S + "test_uniform_flow_preserved_bitwise_2d", S + "test_2d_reproduces_1d_on_y_uniform_data"]),
    ("linear weight d_2 of Sec. 3.3", "4.0 / 49.0, 7.0 / 98.0", "5.0 / 49.0, 7.0 / 98.0",
     [R + "test_weno_smooth_limit_and_zref_order"]),
    ("right state: slope not mirrored", "*val = v; *hslope = -sl;", "*val = v; *hslope = sl;",
     [R + "test_right_state_is_mirror_of_left"]),
    ("half-line first moment: sign of the Gaussian term", "out[1] = U * out[0] + e;", "out[1] = U * out[0] - e;",
     [K + "test_half_line_moments_quadrature"]),
    ("moment recurrence: off-by-one factor", "(n + 1) / (2.0 * lam) * out[n]", "n / (2.0 * lam) * out[n]",
     [K + "test_whole_line_moments_gauss_hermite"]),
    ("<xi^4> of the internal degrees of freedom", "(K * K + 2.0 * K)", "(K * K + K)",
     [K + "test_psi_moment_assembly"]),
    ("energy component of psi: factor 1/2 dropped (1D)",
     "p->coef[0] = p->coef[1] = 0.5; p->a[0] = 2; p->c[1] = 1;",
     "p->coef[0] = p->coef[1] = 1.0; p->a[0] = 2; p->c[1] = 1;", [K + "test_psi_moment_assembly"]),
    ("internal degrees of freedom: the 1D value used in 2D", ": (4.0 - 2.0 * gamma) / (gamma - 1.0);",
     ": (3.0 - gamma) / (gamma - 1.0);", [K + "test_gks_point_euler_limit", S + "test_2d_reproduces_1d_on_y_uniform_data"]),
    ("time integral coefficient of (T2 + T1): sign", "double c3 = -tau * D_;", "double c3 = tau * D_;",
     [V + "test_entropy_wave_decays_at_alpha_k2", C + "test_characteristic_shock_tubes"]),
    ("time integral coefficient of (T2 - Th): sign inside", "tau * (D_ + tau) * e", "tau * (D_ - tau) * e",
     [S + "test_shock_tube_vs_exact_riemann"]),
    ("flux time slope F_t: factor 2 dropped", "4.0 * (o->S1[k] - 2.0 * o->S2[k])", "4.0 * (o->S1[k] - o->S2[k])",
     [S + "test_table1_eighth_order_small_dt"]),
    ("S2O4 second stage: weight dt^2/3 -> dt^2/6 (1D)", "W[k * nx + i] = R[k * nx + i] - dt * dt / 3.0 *",
     "W[k * nx + i] = R[k * nx + i] - dt * dt / 6.0 *", [S + "test_table3_fourth_order_at_cfl_08"]),
    ("Euler energy flux: pressure work dropped (1D)", "F[2] = jmul(U, jadd(E, p));", "F[2] = jmul(U, E);",
     [K + "test_euler_time_derivatives_match_symbolic"]),
    ("second time derivative: the tangential flux dropped",
     "Wtt[k] = -F[k].h[0][2] - (D == 2 ? G[k].h[1][2] : 0.0);", "Wtt[k] = -F[k].h[0][2];",
     [K + "test_euler_time_derivatives_match_symbolic"]),
    ("viscous collision time: mu/rho for mu/p", "P->mu / p :", "P->mu / rho :",
     [V + "test_entropy_wave_decays_at_alpha_k2"]),
    ("collision time: pressure-jump term dropped", "P->c_tau * fabs((pl - pr) / (pl + pr)) * dt",
     "0.0 * fabs((pl - pr) / (pl + pr)) * dt",
     [K + "test_collision_time_pressure_jump_limits", S + "test_pressure_jump_collision_time_damps_shock_oscillations"]),
    ("two-point Gauss rule along the face: wrong node", "const double g = 1.0 / (2.0 * sqrt(3.0));",
     "const double g = 1.0 / (2.0 * sqrt(2.0));", [S + "test_isentropic_vortex_convergence"]),
    ("tangential derivative not divided by the spacing", "in.W0t[k] = dp / ht;", "in.W0t[k] = dp;",
     [S + "test_isentropic_vortex_convergence"]),
    ("tangential WENO-Z reference: wrong candidate", "double Z = fabs(beta[0] - beta[nc - 1]);",
     "double Z = fabs(beta[0] - beta[1]);", [T + "test_jump_value_stays_on_the_smooth_side_and_mirror_symmetry"]),
    ("y-faces: momentum components not rotated", "return (k == 1) ? 2 : (k == 2) ? 1 : k;", "return k;",
     [S + "test_transpose_symmetry"]),
    ("y-faces: x-gradients used as the normal ones", "int gn = (o == 0) ? 1 : 2;", "int gn = 1;",
     [S + "test_transpose_symmetry"]),
    ("characteristic basis: U+c column energy entry", "R[(nv - 1) * nv + nv - 1] = H + U * c;",
     "R[(nv - 1) * nv + nv - 1] = H - U * c;", [C + "test_eigenbasis_diagonalises_the_flux_jacobian"]),
    ("6th-order variant: one linear weight", "8.0 / 70.0", "9.0 / 70.0",
     [X + "test_weights_recombine_printed_candidates_into_the_degree5_fit"]),
    ("viscous time-step bound: half the diffusion term (x)", "2.0 * nu / P->dx", "nu / P->dx",
     [V + "test_viscous_cfl_term"]),
    ("half-step interface state: dt^2/8 -> dt^2/4", "0.125 * dt * dt * o->Wtt[k]", "0.25 * dt * dt * o->Wtt[k]",
     [S + "test_table3_fourth_order_at_cfl_08"]),
    ("non-equilibrium interface part: -t W_t dropped", "- in->W0[k] - t * out->Wt[k]);", "- in->W0[k]);",
     [K + "test_gks_point_equal_states"]),
    ("2D first stage: sign of the y flux difference",
     "- ((0.5 * dt * yr->Fb[k] + 0.125 * dt * dt * yr->Ft[k])",
     "+ ((0.5 * dt * yr->Fb[k] + 0.125 * dt * dt * yr->Ft[k])", [S + "test_transpose_symmetry"]),
    # boundaries
    ("2D x-walls: parity of the x-gradients dropped",
     "int odd = (grp == 0 && var == 1) || (grp == 1 && var != 1) || (grp == 2 && var == 1);",
     "int odd = (grp == 0 && var == 1) || (grp == 2 && var == 1);",
     [S + "test_reflecting_walls_equal_the_mirrored_periodic_domain"]),
    ("2D y-walls: parity of the y-gradients inverted", "(grp == 2 && var != 2);", "(grp == 2 && var == 2);",
     [S + "test_reflecting_walls_equal_the_mirrored_periodic_domain"]),
    ("1D walls: parity of the gradients dropped", "int odd = (grp == 0 && var == 1) || (grp == 1 && var != 1);\n",
     "int odd = (grp == 0 && var == 1);\n", [S + "test_reflecting_walls_equal_the_mirrored_periodic_domain"]),
    ("1D outflow: the normal gradient copied instead of zeroed",
     "else v = (grp == 1) ? 0.0 : E[p * X + (side ? nx - 1 : 0) + NG];", "else v = E[p * X + (side ? nx - 1 : 0) + NG];",
     [T + "test_strong_normal_shock_on_a_2d_grid"]),
    ("2D periodic wrap in x: off by one", "side ? m % nx : ((nx - 1 - m) % nx + nx) % nx",
     "side ? m % nx : ((nx - m) % nx + nx) % nx", [S + "test_2d_reproduces_1d_on_y_uniform_data"]),
    ("2D inflow: the other side's state", "v = (grp == 0) ? inflow_cons[side][var] : 0.0;",
     "v = (grp == 0) ? inflow_cons[1 - side][var] : 0.0;", [S + "test_supersonic_inflow_keeps_its_uniform_state"]),
    # characteristic variables, tangential profiles, scalings
    ("characteristic back-projection: R transposed", "vl[k] += R[k * nv + m] * cvl[m];",
     "vl[k] += R[m * nv + k] * cvl[m];", [C + "test_characteristic_shock_tubes"]),
    ("tangential profile: second-derivative factor", "cc += m * (m - 1) * c[m] * ipow(eta, m - 2);",
     "cc += m * m * c[m] * ipow(eta, m - 2);", [T + "test_segment_profiles_exact_for_polynomials"]),
    ("tangential second derivative divided by h once", "in.W0tt[k] = d2p / (ht * ht);", "in.W0tt[k] = d2p / ht;",
     [S + "test_scale_invariance"]),
    ("tangential slope of the left state not divided by h", "in.Wlt[k] = dw / ht;", "in.Wlt[k] = dw;",
     [S + "test_scale_invariance"]),
    ("mixed derivative not divided by h", "in.W0nt[k] = dp / ht;", "in.W0nt[k] = dp;", [S + "test_scale_invariance"]),
    ("tangential linear weight: wrong candidate", "d[nc - 1] = wfl / wcl;", "d[nc - 1] = wfl / wc0;",
     [S + "test_transpose_symmetry"]),
    # time step, updates, fluxes, moments
    ("2D time step: the y bound ignored", "if (dy < d) d = dy;", "(void)dy;", [V + "test_viscous_cfl_term"]),
    ("time step: sound speed without gamma", "double a = sqrt(P->gamma * p / rho);", "double a = sqrt(p / rho);",
     [S + "test_cfl_rule_reproduces_tam_webb_step_count"]),
    ("1D gradient update: sign", "Ws[(3 + k) * nx + i] = (Rf->Wm[k] - L->Wm[k]) / dx;",
     "Ws[(3 + k) * nx + i] = (L->Wm[k] - Rf->Wm[k]) / dx;", [S + "test_table1_eighth_order_small_dt"]),
    ("2D second stage: sign of the y-gradient term", "W[(8 + k) * PL + c] = R[(8 + k) * PL + c] + dt * dt / 3.0 *",
     "W[(8 + k) * PL + c] = R[(8 + k) * PL + c] - dt * dt / 3.0 *", [S + "test_transpose_symmetry"]),
    ("Euler y-momentum flux: pressure dropped", "G[2] = jadd(jmul(n, V), p);", "G[2] = jmul(n, V);",
     [K + "test_euler_time_derivatives_match_symbolic"]),
    ("energy component of psi: v^2 dropped (2D)",
     "p->coef[0] = p->coef[1] = p->coef[2] = 0.5; p->a[0] = 2; p->b[1] = 2; p->c[2] = 1;",
     "p->coef[0] = p->coef[1] = p->coef[2] = 0.5; p->a[0] = 2; p->c[2] = 1;", [K + "test_psi_moment_assembly"]),
    ("half-line zeroth moment: sign of the erfc argument", "out[0] = 0.5 * erfc(-s * U);",
     "out[0] = 0.5 * erfc(s * U);", [K + "test_half_line_moments_quadrature"]),
    ("time integral coefficient of F0", "double c1 = D_ - tau * (1.0 - e);", "double c1 = D_ - tau * e;",
     [K + "test_gks_point_equal_states"]),
    ("time integral coefficient of Fh", "double c5 = tau * (1.0 - e);", "double c5 = tau * e;",
     [K + "test_gks_point_equal_states"]),
    ("non-equilibrium interface part: sign of the slope term", "NE[k] = e * ((Wh[k] - t * Wsl[k])",
     "NE[k] = e * ((Wh[k] + t * Wsl[k])", [K + "test_gks_point_equal_states"]),
    ("end-of-step interface state: dt^2/6 -> dt^2/2", "dt * dt / 6.0 * o->Wtt[k]", "dt * dt / 2.0 * o->Wtt[k]",
     [S + "test_table3_fourth_order_at_cfl_08"]),
    ("mean flux of the step: factor 4 -> 2", "(4.0 * o->S2[k] - o->S1[k]) / dt", "(2.0 * o->S2[k] - o->S1[k]) / dt",
     [S + "test_shock_tube_vs_exact_riemann"]),
    ("2D y-outflow: the normal gradient copied instead of zeroed",
     "else { int src = side ? ny - 1 : 0; v = (grp == 2) ? 0.0 : AT(p, src, i); }",
     "else { int src = side ? ny - 1 : 0; v = AT(p, src, i); }", [T + "test_strong_normal_shock_along_y_on_a_2d_grid"]),
    ("tangential spacing of x-faces and y-faces exchanged", "double ht = (o == 0) ? P->dy : P->dx;",
     "double ht = (o == 0) ? P->dx : P->dy;", [S + "test_isentropic_vortex_convergence_on_tall_cells"]),
    ("normal second derivative divided by h once", "out->NN[k] = lin[2] / (h * h);", "out->NN[k] = lin[2] / h;",
     [S + "test_scale_invariance"]),
    ("W0nn taken from the wrong row", "in.W0nn[k] = rr[2]->NN[k];", "in.W0nn[k] = rr[1]->NN[k];",
     [S + "test_reflecting_walls_equal_the_mirrored_periodic_domain"]),
    ("right normal slope taken from the left state", "out->Rn[k] = sr[k] / h;", "out->Rn[k] = sl[k] / h;",
     [S + "test_2d_reproduces_1d_on_y_uniform_data"]),
    ("time step: CFL number not applied", "return P->cfl * best;", "return best;",
     [S + "test_table3_fourth_order_at_cfl_08"]),
    ("last step not clipped to t_end", "if (t_end > 0.0 && *t + dt > t_end) dt = t_end - *t;", "(void)0;",
     [S + "test_shock_tube_vs_exact_riemann"]),
    ("Taylor-jet product: one cross term of the Hessian", "a.g[i] * b.g[j] + a.g[j] * b.g[i] + a.h[i][j] * b.v;",
     "a.g[i] * b.g[j] + a.h[i][j] * b.v;", [K + "test_euler_time_derivatives_match_symbolic"]),
    ("Taylor-jet reciprocal: factor 2 of the Hessian", "+ 2.0 * q * q * q * a.g[i] * a.g[j];",
     "+ q * q * q * a.g[i] * a.g[j];", [S + "test_shock_tube_vs_exact_riemann"]),
    ("pressure: kinetic energy without 1/2", "double ke = 0.5 * (*rho) * ((*U) * (*U) + (*V) * (*V));",
     "double ke = (*rho) * ((*U) * (*U) + (*V) * (*V));", [S + "test_transpose_symmetry"]),
    ("1D normal second derivative divided by h once", "in.W0nn[k] = lin[2] / (h * h);", "in.W0nn[k] = lin[2] / h;",
     [S + "test_shock_tube_vs_exact_riemann"]),
    ("1D right normal slope not divided by h", "in.Wr[k] = vr[k]; in.Wrn[k] = sr[k] / h;",
     "in.Wr[k] = vr[k]; in.Wrn[k] = sr[k];", [S + "test_scale_invariance"]),
    ("y-momentum component of psi: u for v",
     "else if (D == 2 && k == 2) { p->n = 1; p->coef[0] = 1.0; p->b[0] = 1; }",
     "else if (D == 2 && k == 2) { p->n = 1; p->coef[0] = 1.0; p->a[0] = 1; }",
     [S + "test_uniform_flow_preserved_bitwise_2d"]),
    ("1D inflow: the other side's state", "else if (bc == BC_INFLOW) v = (grp == 0) ? ic[side][var] : 0.0;",
     "else if (bc == BC_INFLOW) v = (grp == 0) ? ic[1 - side][var] : 0.0;",
     [S + "test_supersonic_inflow_keeps_its_uniform_state"]),
    ("right-state mirror: two slopes exchanged",
     "double m[8] = {s[3], s[2], s[1], s[0], -s[7], -s[6], -s[5], -s[4]};",
     "double m[8] = {s[3], s[2], s[1], s[0], -s[6], -s[7], -s[5], -s[4]};", [S + "test_density_wave_100_cells"]),
]


def _pytest(nodeids, lib, threads):
    env = dict(os.environ, CGKS_ORACLE_LIB=lib, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-m", "pytest", *nodeids, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=REPO, env=env, capture_output=True, text=True, timeout=1200)
    return r.returncode, r.stdout[-3000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    d = tmp_path_factory.mktemp("planted")
    with open(O._SRC) as f:
        src = f.read()

    def job(idx):
        if idx < 0:
            text, ids, threads = src, sorted({n for m in MUTANTS for n in m[3]}), 4
        else:
            _, old, new, ids = MUTANTS[idx]
            assert src.count(old) == 1, f"planting site no longer unique in the oracle source: {old!r}"
            text, threads = src.replace(old, new), 1
        c = os.path.join(d, f"m{idx + 1}.c")
        so = os.path.join(d, f"m{idx + 1}.so")
        with open(c, "w") as f:
            f.write(text)
        O.compile_to(c, so)
        return _pytest(ids, so, threads)

    workers = max(2, min(8, os.cpu_count() or 2))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(job, [-1] + list(range(len(MUTANTS)))))
    return {"control": res[0], "mutants": res[1:]}


def test_unplanted_copy_passes_every_named_pin(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("idx", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(outcomes, idx):
    rc, out = outcomes["mutants"][idx]
    # exit status 1: tests ran and at least one failed (not a collection or usage error)
    assert rc == 1 and " failed" in out, (MUTANTS[idx][0], rc, out)
