"""Mutation check of the oracle's pins: plausible one-line mistakes are planted
in copies of the oracle's C source, each copy is compiled, and the pins that
cover the mistaken part must fail on it.  This is how the pins are known to
pin: a dropped term, a wrong sign, a transposed operand or a wrong index
anywhere in the method's arithmetic changes a result some pin checks.

The mistakes are planted only in throw-away copies under pytest's temporary
directory; the oracle itself is not touched.  CPU only.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

import test_oracle_force
import test_oracle_pins as pins
from oracle import oracle as O

MODULES = {"pins": pins, "force": test_oracle_force}

SRC = os.path.join(os.path.dirname(O.__file__), "lbm_oracle.c")

# name -> (the part of the method it breaks, original text, mistaken text, pins
# as (test name, arguments), a name from test_oracle_force as "force:test");
# each original text occurs exactly once.
MUTANTS = {
    "d2q5_weights": (
        "D2Q5 weights (reading: w0 = 1/3 from cs^2 = 1/3)",
        "1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0", "0.4, 0.15, 0.15, 0.15, 0.15",
        [("test_phase_field_distributions_meet_appendix_a", ())]),
    "d2q9_row_transposed": (
        "Eq. B.2, the c_x^2 c_y row written as c_x c_y^2",
        "M[6 * 9 + i] = cx * cx * cy;", "M[6 * 9 + i] = cx * cy * cy;",
        [("test_d2q9_M_is_the_printed_matrix", ())]),
    "lambda_operands_swapped": (
        "Lambda = M^-1 S M built as M S M^-1",
        "acc += Minv[i * n + k] * S[k] * M[k * n + j];", "acc += M[i * n + k] * S[k] * Minv[k * n + j];",
        [("test_d2q5_lambda_is_the_printed_matrix", (1.0, 1.3, 1.0))]),
    "G_phi_sign": (
        "Eq. 14, sign of the anisotropic source G^phi",
        "out[i] = -W5[i] * (C5[i][0] * Nx", "out[i] = W5[i] * (C5[i][0] * Nx",
        [("test_phase_field_distributions_meet_appendix_a", ())]),
    "n_eq_rest_sign": (
        "Eq. 19, rest population of n^eq",
        "out[0] = C + (W5[0] - 1.0) * qU;", "out[0] = C + (W5[0] + 1.0) * qU;",
        [("test_solute_distributions_meet_appendix_a", ())]),
    "h_eq_dropped_cs2": (
        "Eq. 25, cs^2 dropped from the second-order term",
        "(cu * cu - CS2 * uu)", "(cu * cu - uu)",
        [("test_flow_equilibrium_moments_are_the_printed_ones", (0,))]),
    "dadx_sign": (
        "Eq. 3, sign of d a_s / d(d_x phi)",
        "double dax = 16.0 * eps * px * py * py * (px * px - py * py)",
        "double dax = 16.0 * eps * px * py * py * (py * py - px * px)",
        [("test_anisotropic_vector_is_the_derivative_of_a_s", (0,))]),
    "grain_rotation_sign": (
        "rotation into the crystal frame",
        "double py = -s * gx + c * gy;", "double py = s * gx + c * gy;",
        [("test_anisotropy_rotates_with_the_grain", ())]),
    "Q_single_factor": (
        "Eq. 5, (1 - phi^2)^2 written as (1 - phi^2)",
        "return phi * w - lambda * (theta + Mc * U) * w * w;", "return phi * w - lambda * (theta + Mc * U) * w;",
        [("test_quasi_uniform_phase_field_follows_the_discrete_recurrence", ())]),
    "dtF_sign": (
        "Eq. 13, sign of the 1/2 a_s^2 d_t F term",
        "fs[i] += F[i] + 0.5 * as2 * dF[i];", "fs[i] += F[i] - 0.5 * as2 * dF[i];",
        [("test_quasi_uniform_phase_field_follows_the_discrete_recurrence", ())]),
    "plain_phi_streaming": (
        "Eq. 13 / Remark 2, modified streaming replaced by plain streaming",
        "s->f2[i * N + d] = (fs[i] - (1.0 - as2) * s->f[i * N + d]) / as2;", "s->f2[i * N + d] = fs[i];",
        [("test_anisotropic_planar_front_relaxes_with_a_s_squared", ())]),
    "s1_phi_with_a_s": (
        "Sec. 3.1, a_s instead of a_s^2 in the phase-field relaxation rate",
        "const double s1phi = 1.0 / (as2 * s->kappa0 / CS2 + 0.5);",
        "const double s1phi = 1.0 / (as * s->kappa0 / CS2 + 0.5);",
        [("test_anisotropic_planar_front_relaxes_with_a_s_squared", ())]),
    "J_at_sign": (
        "Eq. 7, sign of the anti-trapping current",
        "double a = -1.0 / (2.0 * sqrt(2.0)) * s->W", "double a = 1.0 / (2.0 * sqrt(2.0)) * s->W",
        [("test_planar_isothermal_front_follows_the_stefan_solution_without_solute_trapping", ())]),
    "grad_q_sign": (
        "Eq. 19, sign of grad q~ = -grad(phi)/2",
        "U, -0.5 * gx, -0.5 * gy, Jx, Jy,", "U, 0.5 * gx, 0.5 * gy, Jx, Jy,",
        [("test_planar_isothermal_front_follows_the_stefan_solution_without_solute_trapping", ())]),
    "J_at_times_D": (
        "Eq. 19, J_at / D written as J_at D",
        "double vx = dCux / CS2 + U * gqx + Jx / D;", "double vx = dCux / CS2 + U * gqx + Jx * D;",
        [("test_planar_isothermal_front_follows_the_stefan_solution_without_solute_trapping", ())]),
    "theta_latent_sign": (
        "Eq. 23, theta = H - h/2 instead of H + h/2",
        "double theta = H + latent(s) * h_of_phi(s->P.h_kind, phi);",
        "double theta = H - latent(s) * h_of_phi(s->P.h_kind, phi);",
        [("test_isothermal_mode_keeps_theta_and_latent_mode_releases_heat", ())]),
    "g_eq_latent_sign": (
        "Eq. 22, sign of the latent term of g_0^eq",
        "out[0] = W5[0] * theta - Lh;", "out[0] = W5[0] * theta + Lh;",
        [("test_isothermal_mode_keeps_theta_and_latent_mode_releases_heat", ())]),
    "u_without_half": (
        "Eq. 26, the 1/2 of u = u* + [1 - q~] f / 2 dropped",
        "*ux = usx + 0.5 * (1.0 - qt) * (*fsx);", "*ux = usx + (1.0 - qt) * (*fsx);",
        [("test_interface_forcing_halves_the_momentum_each_step", ())]),
    "F_u_unweighted": (
        "Eq. 25, the fluid-solid force in F' without its [1 - q~] weight",
        "orc_F_u(Fx + (1.0 - qt) * fsx, Fy + (1.0 - qt) * fsy, Fu);", "orc_F_u(Fx + fsx, Fy + fsy, Fu);",
        [("test_interface_forcing_halves_the_momentum_each_step", ()),
         ("test_solid_stops_the_flow_in_one_step", ())]),
    "pressure_scale": (
        "Eq. 26, cs^2 dropped from the pressure",
        "*p = CS2 / (1.0 - W9[0])", "*p = 1.0 / (1.0 - W9[0])",
        [("test_shear_wave_decays_at_the_viscous_rate", ()),
         ("test_inflow_outflow_channel_becomes_plug_flow", ())]),
    "buoyancy_sign": (
        "reading of the external force: sign of the thermal buoyancy",
        "s->gbT * (theta - s->P.theta_ref)", "s->gbT * (s->P.theta_ref - theta)",
        [("test_warm_melt_rises_and_symmetry_walls_stop_normal_flow", ())]),
    "nee_equilibrium_only": (
        "Guo's extrapolation without the non-equilibrium part",
        "for (int i = 0; i < 9; ++i) s->h2[i * N + b] = eb[i] + s->h2[i * N + f] - ef[i];",
        "for (int i = 0; i < 9; ++i) s->h2[i * N + b] = eb[i];",
        [("test_poiseuille_flow_converges_at_second_order", ())]),
    "side_symmetry_wall": (
        "symmetry walls at x = 0, nx - 1 keeping the normal velocity",
        "ubx = (side < 2) ? 0.0 : mf.ux;", "ubx = mf.ux;",
        [("test_symmetry_side_walls_stop_normal_flow", ())]),
    "stencil_scale": (
        "reading R4, the 1/cs^2 of the nine-point stencil dropped",
        "        gx /= CS2;\n        gy /= CS2;\n", "",
        [("test_stencil_gradient_is_the_nine_point_symbol", ())]),
    "stencil_transposed": (
        "reading R4, neighbour offsets transposed",
        "double ph = s->phi[stencil_index(s, x + C9[i][0], y + C9[i][1])];",
        "double ph = s->phi[stencil_index(s, x + C9[i][1], y + C9[i][0])];",
        [("test_stencil_gradient_is_the_nine_point_symbol", ())]),
    "Cu_history_dropped": (
        "Eq. 19, the backward difference of C u without its previous value",
        "s->Cu_prev[idx] = s->C[idx] * usx;", "s->Cu_prev[idx] = 0.0;",
        [("test_scalar_models_advect_with_the_flow", (0.1, 1))]),
    "h_kind1_coefficient": (
        "Sec. 2, the second h(phi) with 2 phi^3/3 written phi^3/3",
        "return 15.0 / 8.0 * (phi - 2.0 * p3 / 3.0 + p3 * phi * phi / 5.0);",
        "return 15.0 / 8.0 * (phi - p3 / 3.0 + p3 * phi * phi / 5.0);",
        [("test_second_interpolation_function_releases_heat_by_its_closed_form", ())]),
    "local_grad_anisotropy_sign": (
        "Sec. 3.1, sign of the anisotropic term in the local grad(phi) scheme",
        "gx = -s1 / CS2 * (jx + s->kappa0 * nx_);",
        "gx = -s1 / CS2 * (jx - s->kappa0 * nx_);",
        [("force:test_local_gradient_scheme_matches_stencil", ())]),
    "nsub_velocity_scale": (
        "Sec. 4, two-time-scaling: the scalars seeing the flow lattice's velocity, not n_sub times it",
        "s->nsub_scale = (double)P->n_sub;", "s->nsub_scale = 1.0;",
        [("test_scalar_models_advect_with_the_flow", (0.02, 2))]),
    "dirichlet_solute_zero_gradient": (
        "Sec. 4.4's far field: the solute on Dirichlet walls copied from the interior",
        "        Cb = C_of_U(Ub, phib, k);\n", "        Cb = mf.C;\n",
        [("test_dirichlet_walls_give_the_heat_equation_series_solution", ())]),
    "solutal_buoyancy_sign": (
        "reading of the external force: sign of the solutal buoyancy",
        "s->gbC * (C - s->P.C_ref)", "s->gbC * (s->P.C_ref - C)",
        [("test_solute_rich_melt_moves_with_the_sign_of_the_solutal_coefficient", ())]),
    "dirichlet_phi_zero_gradient": (
        "Sec. 4.4's far field: phi on Dirichlet walls copied from the interior",
        "        phib = s->P.dir_phi;\n", "",
        [("test_dirichlet_walls_hold_the_far_field_values", ())]),
    "local_grad_rate_with_a_s": (
        "Sec. 3.1, a_s instead of a_s^2 in the local grad(phi) scheme's relaxation rate",
        "const double s1 = 1.0 / (a1 * a1 * s->kappa0 / CS2 + 0.5);",
        "const double s1 = 1.0 / (a1 * s->kappa0 / CS2 + 0.5);",
        [("force:test_local_gradient_scheme_matches_stencil", ())]),
    "C_of_U_sign": (
        "Eq. 20 inverted: sign of the (1 - k) U term",
        "return 0.5 * (1.0 + k - (1.0 - k) * phi) * (1.0 + (1.0 - k) * U);",
        "return 0.5 * (1.0 + k - (1.0 - k) * phi) * (1.0 - (1.0 - k) * U);",
        [("test_initial_supersaturation_round_trips", ())]),
    "U_of_C_sign": (
        "Eq. 20, sign of the (1 - k) phi term",
        "return (2.0 * C / (1.0 + k - (1.0 - k) * phi) - 1.0) / (1.0 - k);",
        "return (2.0 * C / (1.0 + k + (1.0 - k) * phi) - 1.0) / (1.0 - k);",
        [("test_initial_supersaturation_round_trips", ())]),
    "substep_walls_skipped": (
        "Sec. 4, two-time-scaling: no flow wall pass after the flow sub-steps",
        "        apply_boundaries(s, s->f, s->nC, s->g, 1);\n        swap_ptr(&s->h, &s->h2);\n    }\n    s->steps++;",
        "        swap_ptr(&s->h, &s->h2);\n    }\n    s->steps++;",
        [("test_poiseuille_flow_with_flow_substeps_and_flow_only_steps", (2, False)),
         ("test_inflow_outflow_channel_becomes_plug_flow_with_flow_substeps", (2, False))]),
    "substep_walls_stale_scalars": (
        "reading R11 in the flow sub-steps: wall macros from the previous time level's scalar populations",
        "        apply_boundaries(s, s->f, s->nC, s->g, 1);\n        swap_ptr(&s->h, &s->h2);\n    }\n    s->steps++;",
        "        apply_boundaries(s, s->f2, s->n2, s->g2, 1);\n        swap_ptr(&s->h, &s->h2);\n    }\n    s->steps++;",
        [("test_walls_hold_their_velocity_while_the_melt_warms_them", (2, 0, "symmetry")),
         ("test_walls_hold_their_velocity_while_the_melt_warms_them", (3, 0, "noslip"))]),
    "flow_only_walls_skipped": (
        "Sec. 4.1, flow-only steps without the flow wall pass",
        "        apply_boundaries(s, s->f, s->nC, s->g, 1);\n        swap_ptr(&s->h, &s->h2);\n    }\n    return 0;",
        "        swap_ptr(&s->h, &s->h2);\n    }\n    return 0;",
        [("test_poiseuille_flow_with_flow_substeps_and_flow_only_steps", (1, True)),
         ("test_inflow_outflow_channel_becomes_plug_flow_with_flow_substeps", (1, True))]),
    "flow_only_walls_stale_scalars": (
        "reading R11 in flow-only steps: wall macros from the previous time level's scalar populations",
        "        apply_boundaries(s, s->f, s->nC, s->g, 1);\n        swap_ptr(&s->h, &s->h2);\n    }\n    return 0;",
        "        apply_boundaries(s, s->f2, s->n2, s->g2, 1);\n        swap_ptr(&s->h, &s->h2);\n    }\n    return 0;",
        [("test_walls_hold_their_velocity_while_the_melt_warms_them", (1, 20, "symmetry"))]),
}


def _pin(name):
    """A pin by name: `test_x` from the pin module, or `module:test_x`."""
    mod, _, test = name.rpartition(":")
    return getattr(MODULES[mod or "pins"], test)


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    """Compile every mutant (in parallel) with the oracle's own flags."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("oracle_mutants")
    inc = os.path.dirname(SRC)

    def compile_one(name):
        _, old, new, _ = MUTANTS[name]
        assert src.count(old) == 1, f"{name}: the original text is not in the oracle exactly once"
        c, so = d / f"{name}.c", d / f"{name}.so"
        c.write_text(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                        "-ffp-contract=off", "-I", inc, "-o", str(so), str(c), "-lm"], check=True)
        return name, str(so)

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(ex.map(compile_one, MUTANTS))


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_the_mutant(name, mutant_libs, monkeypatch):
    what, _, _, checks = MUTANTS[name]
    monkeypatch.setattr(O, "_LIB_PATH", mutant_libs[name])
    monkeypatch.setattr(O, "_lib", None)
    monkeypatch.setattr(O, "build", lambda force=False: mutant_libs[name])
    failed = []
    for test, args in checks:
        try:
            _pin(test)(*args)
        except AssertionError:
            failed.append(test)
    assert failed, f"no pin caught the mistake in {what}"


def test_unmutated_copy_passes_the_same_pins(tmp_path, monkeypatch):
    """The harness itself: a copy of the oracle compiled the same way, with no
    mistake planted, passes every pin the mutants are checked with."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    so = tmp_path / "copy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                    "-ffp-contract=off", "-I", os.path.dirname(SRC), "-o", str(so), SRC, "-lm"], check=True)
    monkeypatch.setattr(O, "_LIB_PATH", str(so))
    monkeypatch.setattr(O, "_lib", None)
    monkeypatch.setattr(O, "build", lambda force=False: str(so))
    seen = set()
    for _, _, _, checks in MUTANTS.values():
        for test, args in checks:
            if (test, args) not in seen:
                seen.add((test, args))
                _pin(test)(*args)
