"""The oracle's pins catch plausible mistakes: each case plants one mistake (a dropped term, a
wrong sign, a transposed operand or index) in a copy of oracle/mhd_oracle.c, builds it, and
checks that at least one pin fails against the mutant.  Everything runs on the CPU."""
import importlib.util
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mhd_oracle.c")
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import test_oracle_cfl_chem as T_cc  # noqa: E402
import test_oracle_gravity as T_gr  # noqa: E402
import test_oracle_heatcool as T_hc  # noqa: E402
import test_oracle_ions as T_io  # noqa: E402
import test_oracle_physics as T_ph  # noqa: E402
import test_oracle_ppm as T_ppm  # noqa: E402
import test_oracle_riemann as T_rs  # noqa: E402
import test_oracle_step4 as T_s4  # noqa: E402

# (name, text in mhd_oracle.c, replacement)
MUTATIONS = [
    ("ppm_delta_sign", "P.d = qR - qL;", "P.d = qL - qR;"),
    ("step4_eta_normalisation_two", "eta = -(Dp - Dm) / (3.0 * dq2);", "eta = -(Dp - Dm) / (2.0 * dq2);"),
    ("step4_eta_normalisation_six", "eta = -(Dp - Dm) / (3.0 * dq2);", "eta = -(Dp - Dm) / (6.0 * dq2);"),
    ("step4_eta_sign", "eta = -(Dp - Dm) / (3.0 * dq2);", "eta = (Dp - Dm) / (3.0 * dq2);"),
    ("step4_small_jump_gate_tenth", "if (fabs(dq2) - 0.01 * mn <= 0.0 || Dp * Dm > 0.0)",
     "if (fabs(dq2) - 0.1 * mn <= 0.0 || Dp * Dm > 0.0)"),
    ("step4_small_jump_gate_dropped", "if (fabs(dq2) - 0.01 * mn <= 0.0 || Dp * Dm > 0.0)", "if (Dp * Dm > 0.0)"),
    ("step4_inflection_gate_reversed", "if (fabs(dq2) - 0.01 * mn <= 0.0 || Dp * Dm > 0.0)",
     "if (fabs(dq2) - 0.01 * mn <= 0.0 || Dp * Dm < 0.0)"),
    ("step4_inflection_gate_dropped", "if (fabs(dq2) - 0.01 * mn <= 0.0 || Dp * Dm > 0.0)",
     "if (fabs(dq2) - 0.01 * mn <= 0.0)"),
    ("step4_ramp_slope", "double hb = 20.0 * (eta - 0.05);", "double hb = 10.0 * (eta - 0.05);"),
    ("step4_ramp_threshold", "double hb = 20.0 * (eta - 0.05);", "double hb = 20.0 * (eta - 0.1);"),
    ("step4_flattened_quarter", "double qLp = qc - 0.25 * dm0, qRp = qc + 0.25 * dm0;",
     "double qLp = qc - 0.5 * dm0, qRp = qc + 0.5 * dm0;"),
    ("step4_weights_as_printed", "    qL = hb * qLp + (1.0 - hb) * qL;\n    qR = hb * qRp + (1.0 - hb) * qR;",
     "    qL = (1.0 - hb) * qLp + hb * qL;\n    qR = (1.0 - hb) * qRp + hb * qR;"),
    ("slope_factor_dropped", "b = 2.0 * fabs(dp)", "b = fabs(dp)"),
    ("edge_value_sixth_sign", "qR = 0.5 * (q[2] + q[3]) - (dmp - dm0) * SIXTH;",
     "qR = 0.5 * (q[2] + q[3]) + (dmp - dm0) * SIXTH;"),
    ("dod_average_sign", "return P.R - 0.5 * y * (P.d - P.q6 * (1.0 - TWO_THIRDS * y));",
     "return P.R - 0.5 * y * (P.d + P.q6 * (1.0 - TWO_THIRDS * y));"),
    ("right_eigvec_slow_p_sign", "{as * cs, af * cf * by * sg, af * cf * bz * sg, -af * sc * by, -af * sc * bz, as * gp},",
     "{as * cs, af * cf * by * sg, af * cf * bz * sg, -af * sc * by, -af * sc * bz, -as * gp},"),
    ("left_alfven_sign_dropped", "{0.0, -bz * sg * INV_SQRT2, by * sg * INV_SQRT2, bz * isr2, -by * isr2, 0.0},",
     "{0.0, -bz * INV_SQRT2, by * INV_SQRT2, bz * isr2, -by * isr2, 0.0},"),
    ("upwind_sides_swapped", "double qb = (k % 2 == 0) ? avg_right_end(pl[m], y) : avg_left_end(pr[m], y);",
     "double qb = (k % 2 == 1) ? avg_right_end(pl[m], y) : avg_left_end(pr[m], y);"),
    ("energy_flux_term_dropped", "s->fo[3][cr] = pstar * Vn - Bn * (Bn * Vn + Bt1 * Vt1 + Bt2 * Vt2);",
     "s->fo[3][cr] = pstar * Vn - Bn * (Bn * Vn + Bt1 * Vt1);"),
    ("momentum_tension_dropped", "s->fo[0][cr] = pstar - Bn * Bn;", "s->fo[0][cr] = pstar;"),
    ("ct_curl_sign", "double Rb = curl * ih;", "double Rb = -curl * ih;"),
    ("emf_component_transposed", "s->eA[d][cr] = Bn * Vt1 - Bt1 * Vn;", "s->eA[d][cr] = Bn * Vt2 - Bt2 * Vn;"),
    ("eint_source_sign", "R[4] = ((g_cell - 1.0) * s->eint[c]) * (s->acc[4][c] * ih);",
     "R[4] = -((g_cell - 1.0) * s->eint[c]) * (s->acc[4][c] * ih);"),
    ("lagrangian_upwind_reversed", "if (vn >= 0.0) {\n              for (int o = 0; o < 5; ++o) st[o] = q[v][cl + (o - 2) * sd];",
     "if (vn < 0.0) {\n              for (int o = 0; o < 5; ++o) st[o] = q[v][cl + (o - 2) * sd];"),
    ("rk_weights_transposed", "static const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};",
     "static const double RK_A[3] = {0.0, 0.25, 1.0 / 3.0};"),
    ("cfl_fast_speed_dropped", "double D = v + b + c + ca + cs + cf;", "double D = v + b + c + ca + cs;"),
    ("chem_photodissociation_dropped", "r.D = (r.k2 * nH + r.k3 * nH2) + r.k4;", "r.D = (r.k2 * nH + r.k3 * nH2);"),
    ("k1_temperature_power", "double s2 = sqrt(t2);", "double s2 = t2;"),
    ("regularisation_half_dropped", "double kin = 0.5 * m2 / r;", "double kin = m2 / r;"),
    ("regularisation_max_reversed", "if (s->regul_mode != 0 || e > s->eint[c]) s->eint[c] = e;",
     "if (s->regul_mode != 0 || e < s->eint[c]) s->eint[c] = e;"),
    ("regularisation_max_dropped", "if (s->regul_mode != 0 || e > s->eint[c]) s->eint[c] = e;", "s->eint[c] = e;"),
    ("gamma_eff_weights_swapped", "return (5.0 * n1 + 7.0 * nH2) / (3.0 * n1 + 5.0 * nH2);",
     "return (7.0 * n1 + 5.0 * nH2) / (5.0 * n1 + 3.0 * nH2);"),
    ("gamma_eff_electrons_dropped", "double n1 = (rho - rh2 - rhp) + 2.0 * rhp", "double n1 = (rho - rh2 - rhp) + 1.0 * rhp"),
    ("temperature_electrons_dropped", "return p / ((((nH + nH2) + nHp) + ne) * KB_CGS);",
     "return p / (((nH + nH2) + nHp) * KB_CGS);"),
    ("k6_log_base", "double L = log(T * KB_EV)", "double L = log10(T * KB_EV)"),
    ("k7_denominator_sign", "double Q = 1.0 - 0.38 * x", "double Q = 1.0 + 0.38 * x"),
    ("k8_log_base", "- 4.4e-5 * log10(T))", "- 4.4e-5 * log(T))"),
    ("ion_recombination_dropped", "r.D = r.k7 * ne + r.k8 * n;", "r.D = r.k8 * n;"),
    ("ion_update_sign", "double nHpn = nHp + ts * (q.C - q.D * nHp) / (1.0 + ts * q.D);",
     "double nHpn = nHp + ts * (q.C + q.D * nHp) / (1.0 + ts * q.D);"),
    ("ion_clamp_ignores_h2", "if (nHpn > n - 2.0 * nH2n) nHpn = n - 2.0 * nH2n;", "if (nHpn > n) nHpn = n;"),
    ("ion_rk_register_not_saved", "    memcpy(s->rhp0, s->rhp, bytes);\n", ""),
    ("lambda7_psi_electrons", "sqrt(T) / ne;", "sqrt(T) * ne;"),
    ("lambda8_power", "pow(T / 1e4, 0.8)", "pow(T / 1e4, 0.08)"),
    ("gamma5_density", "h.G5 = 1.92e-28 * n;", "h.G5 = 1.92e-28 * nH;"),
    ("lambda6_electrons_dropped", "h.L6 = 2.18e-11 * q.k6 * nH * ne;", "h.L6 = 2.18e-11 * q.k6 * nH;"),
    ("face_b_average_index", "s->b[d][c] = 0.5 * (Bc[d][srclo] + Bc[d][src]);", "s->b[d][c] = Bc[d][src];"),
    ("lambda2_high_T_constant", "3.9e-19 * exp(-6118.0 / T)", "3.9e-19 * exp(-6181.0 / T)"),
    ("lambda2_low_density_exponent", "(pow(nH2, 0.77) + 1.2 * pow(nH, 0.77))", "(pow(nH2, 0.77) + 1.2 * pow(nH, 0.7))"),
    ("gamma1_critical_density_inverted", "h.G1 = 7.2e-12 * r.C / (1.0 + ncr / n);", "h.G1 = 7.2e-12 * r.C / (1.0 + n / ncr);"),
    ("gamma4_energy", "h.G4 = 6.4e-13 * r.k4 * nH2;", "h.G4 = 6.4e-12 * r.k4 * nH2;"),
    ("heatcool_limiter", "if (d < -0.5 * eint) d = -0.5 * eint;", "if (d < -0.25 * eint) d = -0.25 * eint;"),
    ("heatcool_energy_only_total", "        s->E[c] = s->E[c] + d;\n", "        s->E[c] = s->E[c] + 2.0 * d;\n"),
    ("poisson_symbol_factor", "double f = -(2.0 / 3.0) * M_PI * s->grav_g * h * h / (1.0 - cx * cy * cz);",
     "double f = -(1.0 / 3.0) * M_PI * s->grav_g * h * h / (1.0 - cx * cy * cz);"),
    ("poisson_symbol_sign", "double f = -(2.0 / 3.0) * M_PI * s->grav_g * h * h / (1.0 - cx * cy * cz);",
     "double f = (2.0 / 3.0) * M_PI * s->grav_g * h * h / (1.0 - cx * cy * cz);"),
    ("poisson_axis_table", "double cx = (3.0 - 2.0 * si * si) / 3.0, cy", "double cx = (3.0 - 1.0 * si * si) / 3.0, cy"),
    ("gravity_energy_uses_rho", "            R[3] = R[3] + s->m[d][c] * gd;", "            R[3] = R[3] + s->rho[c] * gd;"),
    ("gravity_central_difference", "double gd = -(s->phi[c + ST(s, d)] - s->phi[c - ST(s, d)]) * (0.5 * ih);",
     "double gd = -(s->phi[c + ST(s, d)] - s->phi[c]) * ih;"),
]


def load_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: pattern must occur exactly once"
    csrc = tmp_path / f"{name}.c"
    csrc.write_text(src.replace(old, new))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                    str(csrc), "-lm"], check=True)
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._LIB = str(lib)
    mod.build = lambda force=False: str(lib)
    return mod


def pins(O):
    """A fast selection of the pins, each run against module O."""
    hc = lambda: O.Sim(4, 4, 4, 5.0 / 3.0, 2.0, chem=1, heatcool=1)
    yield "heatcool_branches", lambda: [T_hc.test_lambda2_branches_join(hc(), T, r) for T, r in
                                        [(1087.0, 1e8), (4031.0, 1e-6)]]
    yield "heatcool_limits", lambda: T_hc.test_lambda2_density_limits(hc())
    yield "heatcool_gamma1", lambda: T_hc.test_gamma1_critical_density_limits(O, hc())
    yield "heatcool_gamma4", lambda: T_hc.test_gamma4_per_photodissociation(hc())
    yield "heatcool_step", lambda: T_hc.test_euler_step_is_linear_and_limited(hc())
    yield "heatcool_box", lambda: T_hc.test_box_stage_changes_only_the_energies(O)
    yield "gravity_27pt", lambda: [T_gr.test_potential_satisfies_the_27_point_equation(O, sh) for sh in
                                   [(8, 10, 12), (5, 7, 9)]]
    yield "gravity_stage", lambda: T_gr.test_eulerian_stage_with_gravity_only(O)
    yield "gravity_fall", lambda: T_gr.test_gas_falls_towards_the_density_peak(O)
    io = lambda **kw: O.Sim(4, 4, 4, 5.0 / 3.0, 2.0, chem=1, heatcool=1, ions=1, **kw)
    yield "ions_gamma", lambda: [T_io.test_gamma_eff_is_the_equipartition_value(O, *a) for a in
                                 [(1.0, 0.0, 1.0), (1.0, 0.4, 0.3)]]
    yield "ions_temperature", lambda: T_io.test_temperature_counts_the_particles(O, 300.0, 2.0, 1.0, 0.5)
    yield "ions_k6", lambda: T_io.test_k6_at_one_electron_volt_and_rising(O)
    yield "ions_k6_activation", lambda: T_io.test_k6_activation_energy_is_the_ionisation_potential(O)
    yield "ions_k7", lambda: T_io.test_k7_at_one_kelvin_and_falling_in_hot_gas(O)
    yield "ions_k8", lambda: T_io.test_k8_constant_and_power_law(O)
    yield "ions_terms", lambda: T_io.test_creation_and_destruction_terms(O)
    yield "ions_energy", lambda: T_io.test_energy_per_event(io())
    yield "ions_lambda8", lambda: T_io.test_lambda8_power_laws(io())
    yield "ions_lambda7", lambda: T_io.test_lambda7_electron_scaling(O)
    yield "ions_fixed_point", lambda: T_io.test_ion_equilibrium_is_a_fixed_point(O, io())
    yield "ions_limits", lambda: T_io.test_ion_update_limits(io())
    yield "ions_physical", lambda: T_io.test_species_stay_physical_and_nuclei_are_conserved(O, io())
    yield "ions_lagrangian", lambda: T_io.test_lagrangian_stage_carries_an_exact_ion_fraction(O)
    yield "step4_cubic", lambda: [T_s4.test_eta_and_weight_closed_form_on_a_cubic(O, a) for a in T_s4.A_VALUES]
    yield "step4_parabola", lambda: [T_s4.test_parabola_edges_follow_the_weight(O, a) for a in T_s4.A_VALUES]
    yield "step4_inflection", lambda: [T_s4.test_no_inflection_zeroes_eta(O, b, act) for b, act in
                                       [(2.9, True), (3.1, False), (-3.1, False)]]
    yield "step4_small_jumps", lambda: [T_s4.test_small_jumps_zero_eta(O, 1.0, f, act) for f, act in
                                        [(0.98, True), (1.02, False)]]
    yield "step4_sine", lambda: T_s4.test_sampled_sine_closed_form(O)
    st = T_rs.random_states(5, 7)
    yield "eigen", lambda: [T_rs.test_eigen_identities(O, s, 1e-11) for s in st]
    yield "linear_riemann", lambda: [T_rs.test_flat_riemann_matches_numpy_linear_solution(O, k) for k in range(3)]
    yield "acoustic", lambda: [T_rs.test_acoustic_limit(O, k) for k in range(2)]
    yield "appB", lambda: [T_rs.test_appendix_B_expansion(O, k) for k in range(2)]
    yield "ppm_linear", lambda: T_ppm.test_linear_data_exact_edges(O)
    yield "ppm_average", lambda: T_ppm.test_cell_average_and_endpoints(O)
    yield "ppm_dod", lambda: T_ppm.test_domain_of_dependence_averages_match_quadrature(O)
    yield "cfl", lambda: [T_cc.test_cfl_denominator_closed_form(O, s) for s in
                          [(1.0, [0, 0, 0], [0.75, 1.0, 0.0], 1.0, 2.0)]]
    yield "gamma", lambda: T_cc.test_gamma_eff_limits(O)
    yield "rates", lambda: [T_cc.test_app_d_rates_golden(O, r) for r in T_cc._golden()]
    yield "chem_solver", lambda: T_cc.test_chemistry_update_limits_and_exact_solution(O)
    yield "conservation", lambda: T_ph.test_periodic_conservation_and_div_b(O)
    yield "uniform", lambda: T_ph.test_uniform_state_is_stationary(O)
    yield "regularisation", lambda: T_ph.test_regularisation_restores_the_energy_closure(O)
    yield "regularisation_entropy", lambda: T_ph.test_regularisation_never_lowers_the_entropy(O)
    yield "faces_from_cells", lambda: T_ph.test_faces_from_linear_cell_field_are_midpoint_values(O)
    # the whole-run pins last (seconds each): a mutation caught above never runs them
    yield "ot_symmetry", lambda: T_ph.test_orszag_tang_point_symmetry(O)
    yield "sod", lambda: T_ph.test_sod_converges_to_exact_solution(O)
    yield "oblique_waves", lambda: [T_ph.test_oblique_linear_wave_converges(O, k) for k in ["fast", "alfven"]]
    yield "waves", lambda: [T_ph.test_linear_wave_first_order_convergence(O, k) for k in ["fast", "alfven", "slow", "entropy"]]


def first_failing_pin(O):
    for name, fn in pins(O):
        try:
            fn()
        except Exception:  # an assertion, or a non-physical state the oracle reports
            return name
    return None


def test_unmutated_oracle_passes_the_selection(tmp_path):
    O = load_mutant(tmp_path, "none", "#define NG 4", "#define NG 4")
    assert first_failing_pin(O) is None


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(tmp_path, name, old, new):
    O = load_mutant(tmp_path, name, old, new)
    caught = first_failing_pin(O)
    assert caught is not None, f"mutation {name} survived every pin"
