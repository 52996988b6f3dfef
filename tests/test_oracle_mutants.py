"""The oracle's pins must catch plausible mistakes in the oracle.

Each case compiles a copy of the oracle's C source with one planted slip
(on the CPU, into a temporary directory), runs the pin that should reject it
against that copy, and requires the pin to fail.  The committed oracle is
never modified.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

# name: (original text, planted slip, pin expected to fail)
MUTANTS = {
    "guo_term_in_Pi_dropped": (
        "(1.0 - 0.5 / tau) * (u[a] * G[b] + G[a] * u[b])",
        "0.0 * (u[a] * G[b] + G[a] * u[b])",
        "test_collision_matches_bgk_guo_moments"),
    "viscosity_rate_wrong": (
        "Pst[a][b] = Peq + (1.0 - 1.0 / tau) * (Pi[a][b] - Peq)",
        "Pst[a][b] = Peq + (1.0 - 1.1 / tau) * (Pi[a][b] - Peq)",
        "test_collision_matches_bgk_guo_moments"),
    "coriolis_sign": (
        "G[a] = rho * a0[a] + fib[a] - 2.0 * rho * wu[a]",
        "G[a] = rho * a0[a] + fib[a] + 2.0 * rho * wu[a]",
        "test_coriolis_solve_satisfies_eq3"),
    "centrifugal_sign": (
        "a0[a] = -acc[a] - t1[a] - t3[a];", "a0[a] = -acc[a] - t1[a] + t3[a];",
        "test_frame_accel_pure_rotation"),
    "push_instead_of_pull": (
        "int s[3] = {x - C[i][0], y - C[i][1], z - C[i][2]};",
        "int s[3] = {x + C[i][0], y + C[i][1], z + C[i][2]};",
        "test_galilean_advection_direction"),
    "stencil_shifted": (
        "int base = (int)floor(X) - 1;", "int base = (int)floor(X) - 2;",
        "test_ib_interp_reproduces_linear_fields"),
    "delta_outer_branch": (
        "if (r <= 2.0) return (5.0 - 2.0 * r - sqrt",
        "if (r <= 2.0) return (5.0 - 2.0 * r + 0.0*sqrt",
        "test_peskin_phi_golden_values"),
    "torque_cross_order": (
        "cross(r, F, T);", "cross(F, r, T);",
        "test_ib_momentum_and_angular_momentum_balance"),
    "half_force_shift_missing_in_interp": (
        "o->j[3 * c + a] / o->rho[c] + 0.5 * a0[a];",
        "o->j[3 * c + a] / o->rho[c] + 0.0 * a0[a];",
        "test_comoving_markers_feel_no_force"),
    "direct_forcing_factor_1": (
        "dF[3 * l + a] = 2.0 * Ri[3 * l]", "dF[3 * l + a] = 1.0 * Ri[3 * l]",
        "test_stokes_drag_periodic_sphere_array"),
    "mdf_velocity_not_corrected": (
        "ut[3 * c + a] += dfib[3 * c + a] / (2.0 * o->rho[c]);",
        "ut[3 * c + a] += 0.0 * dfib[3 * c + a] / (2.0 * o->rho[c]);",
        "test_multi_direct_forcing_isolated_markers_closed_form"),
    "mdf_full_velocity_shift": (
        "ut[3 * c + a] += dfib[3 * c + a] / (2.0 * o->rho[c]);",
        "ut[3 * c + a] += dfib[3 * c + a] / (1.0 * o->rho[c]);",
        "test_multi_direct_forcing_isolated_markers_closed_form"),
    "segment_ref_ignored": (
        "const double *rs = o->has_seg_ref ? o->seg_ref[sg] : o->ref;",
        "const double *rs = o->ref;",
        "test_segment_reference_points_transport_the_moment"),
    "region_momentum_alpha_unclamped": (
        "if (al > 1.0) al = 1.0;", "if (al > 2.0) al = 1.0;",
        "test_region_momentum_volume_and_inertia"),
    "eq3_wrong_hermite_shift": (
        "CS2 * (c[a] * (b == g) + c[b] * (a == g) + c[g] * (a == b));",
        "CS2 * (c[a] * (b == g) + c[b] * (a == g));",
        "test_third_order_equilibrium_moments"),
    "eq3_post_collision_dropped": (
        "if (eq_order == 3) {   /* the post-collision state carries the equilibrium's third moments */",
        "if (0) {   /* the post-collision state carries the equilibrium's third moments */",
        "test_third_order_equilibrium_restores_galilean_invariance_of_shear_decay"),
    "slip_projection_dropped": (
        "for (int a = 0; a < 3; ++a) dF[3 * l + a] = dn * nl[a];",
        "for (int a = 0; a < 3; ++a) dF[3 * l + a] = dF[3 * l + a] + 0.0 * dn * nl[a];",
        "test_slip_forcing_isolated_markers_closed_form"),
    "slip_tangential_kept": (
        "for (int a = 0; a < 3; ++a) dF[3 * l + a] = dn * nl[a];",
        "for (int a = 0; a < 3; ++a) dF[3 * l + a] = dn * nl[a] + 0.01 * (dF[3 * l + a] - dn * nl[a]);",
        "test_slip_sheet_leaves_tangential_shear_untouched"),
    "mdf_force_not_accumulated": (
        "o->Fm[3 * l + a] += dF[3 * l + a];", "o->Fm[3 * l + a] = dF[3 * l + a];",
        "test_multi_direct_forcing_isolated_markers_closed_form"),
    "freeslip_normal_kept": (
        "if (o->face[fa] == ORC_FREESLIP) ub[a] = 0.0;", "if (0) ub[a] = 0.0;",
        "test_nee_face_values_and_edge_precedence"),
    "outflow_density_extrapolated": (
        "rb = o->rho_out;", "rb = rf;",
        "test_nee_reaches_uniform_inflow_from_rest"),
    "collision_force_shift_dropped": (
        "v[a] = j[a] / rho + 0.5 * a0[a] + fib[a] / (2.0 * rho);",
        "v[a] = j[a] / rho + 0.5 * a0[a] + 0.0 * fib[a] / (2.0 * rho);",
        "test_moving_sphere_and_oncoming_flow_feel_the_same_drag"),
    "marker_velocity_halved": (
        "dF[3 * l + a] = 2.0 * Ri[3 * l] * (o->U[3 * l + a] - Ui[3 * l + a]);",
        "dF[3 * l + a] = 2.0 * Ri[3 * l] * (0.5 * o->U[3 * l + a] - Ui[3 * l + a]);",
        "test_moving_sphere_and_oncoming_flow_feel_the_same_drag"),
    "nee_nonequilibrium_dropped": (
        "o->f[cb * Q + i] = feq[i] + (1.0 - 1.0 / o->tau) * fneq[i];",
        "o->f[cb * Q + i] = feq[i];",
        "test_freeslip_walls_are_exact_for_tangential_shear"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_rejects_planted_slip(name):
    orig, slip, pin = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(orig) == 1, "mutation anchor moved: " + name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "mutant.so")
        open(c, "w").write(src.replace(orig, slip))
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", so, c,
                        "-lm"], check=True)
        env = dict(os.environ, ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", pin],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert "passed" not in r.stdout.splitlines()[-1] or "failed" in r.stdout.splitlines()[-1], \
            r.stdout[-2000:]
        assert r.returncode != 0, "pin %s did not catch %s" % (pin, name)
