"""Plant plausible mistakes in a temporary copy of the oracle and check that
the pins catch every one of them.

Each mutant is compiled from a copy of the oracle sources with one textual
change in oracle.c or born.c (a dropped term, a flipped sign, a wrong index, a
transposed operand, a missing factor); the committed oracle is never touched.
A mutant survives only if all pins of its file (``PINS`` or ``BORN_PINS``)
still pass, which fails the test.
"""
import os
import shutil

import pytest

import oracle
from tests import test_oracle_absorption_pins as apins
from tests import test_oracle_born_bspline_pins as bbpins
from tests import test_oracle_born_pins as bpins
from tests import test_oracle_bspline_pins as spins
from tests import test_oracle_pins as pins
from tests import test_oracle_r13_pins as r13pins

MUTANTS = {
    "rk4_weight": ("2.0 * k2[q] + 2.0 * k3[q]", "k2[q] + 2.0 * k3[q]"),
    "rhs_sign": ("k[2] = -(f[1] - gd * st[2]) / f[0];", "k[2] = (f[1] - gd * st[2]) / f[0];"),
    "rhs_drop_projection": ("k[3] = -(f[2] - gd * st[3]) / f[0];", "k[3] = -(f[2]) / f[0];"),
    "bilinear_transposed_weight": ("S->w[1] = tx * (1 - ty);", "S->w[1] = ty * (1 - tx);"),
    "bilinear_wrong_neighbour": ("S->k[2] = S->k[0] + F->nx;", "S->k[2] = S->k[0] + 1;"),
    "central_difference_scale": ("else F->gx[k] = (F->c[k + 1] - F->c[k - 1]) / (2.0 * h);",
                                 "else F->gx[k] = (F->c[k + 1] - F->c[k - 1]) / h;"),
    "edge_difference_scale": ("if (j == 0) F->gy[k] = (F->c[k + nx] - F->c[k]) / h;",
                              "if (j == 0) F->gy[k] = (F->c[k + nx] - F->c[k]) / (2.0 * h);"),
    "trapezoid_full_last_step": ("T += dsp * 0.5 * (s_prev + f[3]);", "T += ds * 0.5 * (s_prev + f[3]);"),
    "endpoint_correction_sign": ("T += s_prev * corr;", "T -= s_prev * corr;"),
    "endpoint_weight_missing": ("alpha[m] += corr;", "(void)corr;"),
    "landing_no_newton": ("for (int it = 0; it < 2; ++it) {", "for (int it = 0; it < 0; ++it) {"),
    "secant_sign": ("next = ok ? cur.theta - cur.m * (cur.theta - prev.theta) / den : 0.0;",
                    "next = ok ? cur.theta + cur.m * (cur.theta - prev.theta) / den : 0.0;"),
    "orientation_probe_flipped": ("const int ccw = (ep.m / R + psi_r) < M_PI;",
                                  "const int ccw = (ep.m / R + psi_r) > M_PI;"),
    "adjoint_missing_chain": ("g_c[j] = -1000.0 * acc[j] / (c_mps[j] * c_mps[j]);",
                              "g_c[j] = -1000.0 * acc[j] / c_mps[j];"),
    "adjoint_drop_alpha": ("gs[S.k[q]] += g_tof[k] * alpha[m] * S.w[q];",
                           "gs[S.k[q]] += g_tof[k] * S.w[q];"),
    "speed_units": ("F->c[k] = v * 1e-3;", "F->c[k] = v * 1e-2;"),
    "slowness_uses_c": ("f[3] += S.w[q] * F->s[k];", "f[3] += S.w[q] * F->c[k];"),
    "heun_end_slope_only": ("out[q] = st[q] + 0.5 * hs * (k1[q] + k2[q]);", "out[q] = st[q] + hs * k2[q];"),
    "fan_points_angle_off_by_one": ("        t[q] = fan_theta(a_min, step, k);\n",
                                    "        t[q] = fan_theta(a_min, step, k + 1);\n"),
    "fan_inverse_poly_node_dropped": ("if (b != a) l *= (0.0 - m[b]) / (m[a] - m[b]);",
                                      "if (b != a && b != n - 1) l *= (0.0 - m[b]) / (m[a] - m[b]);"),
    "fan_second_angle_without_trace": ("const double m5[5] = {cur.m, m4[0], m4[1], m4[2], m4[3]};",
                                       "const double m5[5] = {prev.m, m4[0], m4[1], m4[2], m4[3]};"),
    "fan_margin_from_fan_step": ("    double margin = ds / R;\n    if (margin < 1e-9) margin = 1e-9;\n"
                                 "    const double a_min = th_lo + margin, a_max = th_hi - margin;\n"
                                 "    const double step = (a_max - a_min) / (K - 1);\n    for (int k = 0; k < K; ++k) {",
                                 "    double margin = fan_ds / R;\n    if (margin < 1e-9) margin = 1e-9;\n"
                                 "    const double a_min = th_lo + margin, a_max = th_hi - margin;\n"
                                 "    const double step = (a_max - a_min) / (K - 1);\n    for (int k = 0; k < K; ++k) {"),
    "fan_traced_at_link_step": ("fan_theta(a_min, step, k), fan_ds, NULL, NULL, 0, &tr);",
                                "fan_theta(a_min, step, k), ds, NULL, NULL, 0, &tr);"),
    "subfan_angles_shifted": ("{ return ta + (tb - ta) * q / (M + 1); }",
                              "{ return ta + (tb - ta) * (q - 1) / (M + 1); }"),
    "subfan_jump_taken_for_a_crossing": ("|| !(fabs(sm[i] - sm[i - 1]) < M_PI * R) ||", "||"),
    "subfan_candidate_ignored": ("if (c3 >= fmin(st[i - 1], st[i]) && c3 <= fmax(st[i - 1], st[i])) j = i;",
                                 "j = i;"),
    "subfan_bracket_orientation": ("const int neg = sm[j - 1] < 0 ? j - 1 : j, nonneg = sm[j - 1] < 0 ? j : j - 1;",
                                   "const int neg = j - 1, nonneg = j;"),
    "subfan_gap_taken_for_a_crossing": ("|| pos[i] != pos[i - 1] + 1)", ")"),
    "subfan_window_with_ends": ("interior[j - 2] && interior[j - 1] && interior[j] && interior[j + 1]) {",
                                "1) {"),
    "subfan_only_rising_cubic": ("if (up || down) {", "if (up) {"),
    "subfan_cubic_point_dropped": ("const double v = inverse_poly_root(st + j - 2, sm + j - 2, 4);",
                                   "const double v = inverse_poly_root(st + j - 2, sm + j - 2, 3);"),
    "subfan_cubic_shifted": ("const double v = inverse_poly_root(st + j - 2, sm + j - 2, 4);",
                             "const double v = inverse_poly_root(st + j - 1, sm + j - 1, 4);"),
    "subfan_start_from_far_end": ("const int lo = fabs(B->fa) <= fabs(B->fb);",
                                  "const int lo = fabs(B->fa) > fabs(B->fb);"),
    "subfan_misfit_sign": ("sm[n] = R * (mod_2pi(atan2(tr.hit[1], tr.hit[0]) - phi_e) - psi_r);",
                           "sm[n] = R * (psi_r - mod_2pi(atan2(tr.hit[1], tr.hit[0]) - phi_e));"),
}

# fast pins first; a mutant is killed by the first pin that fails
PINS = [
    pins.test_subfan_angles_evenly_inside,
    pins.test_subfan_prediction_exact_for_cubic_inverse,
    pins.test_subfan_picks_the_crossing_at_the_plain_candidate,
    pins.test_bilinear_exact_for_bilinear_field,
    pins.test_homogeneous_straight_rays,
    pins.test_path_matrix_invariants,
    pins.test_adjoint_is_transpose,
    pins.test_hits_land_on_ring_and_within_tol,
    lambda orc: pins.test_linear_gradient_closed_form(orc, 1.0),
    pins.test_rk4_fourth_order_on_circular_arc,
    pins.test_heun_second_order_on_circular_arc,
    pins.test_heun_linking_converges_to_analytic_circles,
    pins.test_paper_acoustic_length_experiment,
    pins.test_fisheye_ring_closed_form_converges_h2,
    pins.test_adjoint_matches_central_differences,
    pins.test_fan_start_prediction_accuracy,
    pins.test_fan_step_changes_only_the_predictions,
    pins.test_subfan_refines_only_the_third_angle,
]


BSPLINE_MUTANTS = {
    "bspline_basis_weight": ("b[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;",
                             "b[1] = (3.0 * t * t * t - 6.0 * t * t + 3.0) / 6.0;"),
    "bspline_basis_swapped": ("b[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;",
                              "b[2] = (-3.0 * t * t * t + 3.0 * t * t - 3.0 * t + 1.0) / 6.0;"),
    "bspline_derivative_no_h": ("S->wx[q] = dbx[a] * by[b] / F->h;", "S->wx[q] = dbx[a] * by[b];"),
    "bspline_derivative_wrong_axis": ("S->wy[q] = bx[a] * dby[b] / F->h;", "S->wy[q] = dbx[a] * by[b] / F->h;"),
    "bspline_boundary_not_mirrored": ("static double bs_sup(int i, int n) { return i == 0 ? 2.0 / 6.0 : 1.0 / 6.0; }",
                                      "static double bs_sup(int i, int n) { return i == 0 ? 1.0 / 6.0 : 1.0 / 6.0; }"),
    "bspline_prefilter_x_only": ("for (int i = 0; i < nx; ++i) bs_solve_1d(ny, a + i, (size_t)nx, transpose, cp);",
                                 ";"),
    "bspline_index_clamped": ("if (v > n - 1) v = 2 * (n - 1) - v;", "if (v > n - 1) v = n - 1;"),
    "bspline_slowness_from_c": ("f[3] += S.w[q] * F->as[k];", "f[3] += S.w[q] / F->ac[k];"),
    "bspline_adjoint_not_transposed": ("if (g_interp == 1 && bspline_coef(F.nx, F.ny, acc, acc, 1)) bad = 1;",
                                       "if (g_interp == 1 && bspline_coef(F.nx, F.ny, acc, acc, 0)) bad = 1;"),
    "bspline_adjoint_no_prefilter": ("if (g_interp == 1 && bspline_coef(F.nx, F.ny, acc, acc, 1)) bad = 1;",
                                     "if (0 && bspline_coef(F.nx, F.ny, acc, acc, 1)) bad = 1;"),
    "bspline_transpose_sub": ("sub = transpose ? bs_sup(i - 1, n) : bs_sub(i, n);",
                              "sub = transpose ? bs_sup(i, n) : bs_sub(i, n);"),
}


def _in_bspline(pin):
    def run(orc):
        with orc.interpolator("bspline"):
            pin(orc)
    return run


BSPLINE_PINS = [_in_bspline(p) for p in (
    spins.test_bspline_coefficients,
    spins.test_bspline_samples_match_scipy_everywhere,
    spins.test_bspline_reproduces_cubics_with_exact_gradient,
    spins.test_bspline_is_c2_across_cell_edges,
    spins.test_bspline_gradient_is_the_derivative_of_the_value,
    spins.test_bspline_homogeneous_straight_rays,
    spins.test_bspline_path_matrix_and_adjoint,
    lambda orc: spins.test_bspline_linear_gradient_closed_form(orc, 1.0),
    spins.test_bspline_paper_radius_experiment,
    spins.test_bspline_fisheye_ring_closed_form,
)]


BORN_MUTANTS = {
    "born_abs_path_in_mm": ("const double L = p.L + 1e-3 * ds * 0.5 * (p.al + f[F_AL]);",
                            "const double L = p.L + ds * 0.5 * (p.al + f[F_AL]);"),
    "born_abs_left_rule": ("const double L = p.L + 1e-3 * ds * 0.5 * (p.al + f[F_AL]);",
                           "const double L = p.L + 1e-3 * ds * p.al;"),
    "born_abs_extrapolation_sign": ("const double L = p->L + 1e-3 * p->al * along;",
                                    "const double L = p->L - 1e-3 * p->al * along;"),
    "born_abs_no_extrapolation": ("const double L = p->L + 1e-3 * p->al * along;", "const double L = p->L;"),
    "born_abs_gain": ("const double amp = A * exp(-wy * L);", "const double amp = A * exp(wy * L);"),
    "born_abs_omega_per_us": ("return pow(2.0 * M_PI * f_mhz * 1e6, y);", "return pow(2.0 * M_PI * f_mhz, y);"),
    "born_abs_linear_law": ("return pow(2.0 * M_PI * f_mhz * 1e6, y);", "return pow(2.0 * M_PI * f_mhz * 1e6, 1.0);"),
    "born_abs_adjoint_lossless": ("const double wy = Lam ? omega_pow(f_mhz[f], y) : 0.0;\n                for",
                                  "const double wy = 0.0;\n                for"),
    "born_drop_cnn": ("k[5] = -cnn / (f[F_C] * f[F_C]) * st[4];", "k[5] = 0.0 * cnn;"),
    "born_cnn_sign": ("k[5] = -cnn / (f[F_C] * f[F_C]) * st[4];", "k[5] = cnn / (f[F_C] * f[F_C]) * st[4];"),
    "born_drop_hxy": ("- 2.0 * dx * dy * f[F_HXY]", "- 0.0 * dx * dy * f[F_HXY]"),
    "born_hxx_hyy_swapped": ("(dy * dy * f[F_HXX] - 2.0 * dx * dy * f[F_HXY] + dx * dx * f[F_HYY])",
                             "(dx * dx * f[F_HXX] - 2.0 * dx * dy * f[F_HXY] + dy * dy * f[F_HYY])"),
    "born_hessian_scale": ("F->v[F_HXY][k] = (c[k + nx + 1] - c[k + nx - 1] - c[k - nx + 1] + c[k - nx - 1]) / (4 * h * h);",
                           "F->v[F_HXY][k] = (c[k + nx + 1] - c[k + nx - 1] - c[k - nx + 1] + c[k - nx - 1]) / (2 * h * h);"),
    "born_P0_is_c": ("double st[6] = {xe, ye, cos(theta), sin(theta), 0.0, 1.0 / c_t}",
                     "double st[6] = {xe, ye, cos(theta), sin(theta), 0.0, c_t}"),
    "born_Q_missing_c": ("k[4] = f[F_C] * st[5];", "k[4] = st[5];"),
    "born_amplitude_c_of_transducer": ("const double A = sqrt(p->c / (M->c_t * fabs(clamp_q(Qf, h))));",
                                       "const double A = sqrt(M->c_t / (M->c_t * fabs(clamp_q(Qf, h))));"),
    "born_amplitude_no_sqrt": ("const double A = sqrt(p->c / (M->c_t * fabs(clamp_q(Qf, h))));",
                               "const double A = p->c / (M->c_t * fabs(clamp_q(Qf, h)));"),
    "born_first_order_only": ("p->T + p->s * along + 0.5 * curv * across * across, fabs(across), A, L);",
                              "p->T + p->s * along, fabs(across), A, L);"),
    "born_curvature_at_sample": ("const double Qf = p->Q + along * p->c * p->P;", "const double Qf = p->Q;"),
    "born_amplitude_no_distance_penalty": ("const double score = cand + M->eta * q * q;",
                                           "const double score = cand + 0.0 * q * q;"),
    "born_nearest_node_only": ("for (int i = ic - 1; i <= ic + 1; ++i) {", "for (int i = ic; i <= ic; ++i) {"),
    "born_latest_arrival": ("if (cand < M->T[k]) M->T[k] = cand;",
                            "if (!(cand <= M->T[k]) || M->T[k] == INFINITY) M->T[k] = cand;"),
    "born_T_uses_c": ("const double T = p.T + ds * 0.5 * (p.s + f[F_S]);",
                      "const double T = p.T + ds * 0.5 * (p.c + f[F_C]);"),
    "born_apply_conj": ("sim += (ar * bi + ai * br) * dc[k];", "sim += (ar * bi - ai * br) * dc[k];"),
    "born_apply_omega_not_squared": ("const double scale = omega * omega * g->h * g->h;\n        const double wy = Lam ? omega_pow(f_mhz[f], y) : 0.0;\n#pragma",
                                     "const double scale = omega * g->h * g->h;\n        const double wy = Lam ? omega_pow(f_mhz[f], y) : 0.0;\n#pragma"),
    "born_apply_keeps_diagonal": ("if (e != r && e >= 0", "if (e >= 0"),
    "born_adjoint_conj_one_factor": ("acc += scale * (pr * dd[0] + pi * dd[1]);",
                                     "acc += scale * (pr * dd[0] - pi * dd[1]);"),
    "born_adjoint_uses_diagonal": ("if (r == e) continue;\n                        const double br", "const double br"),
    "born_phase_units": ("const double omega = 2.0 * M_PI * f_mhz[f];\n        const double scale = omega * omega * g->h * g->h;\n        const double wy",
                         "const double omega = M_PI * f_mhz[f];\n        const double scale = omega * omega * g->h * g->h;\n        const double wy"),
}

BORN_PINS = [
    bpins.test_fan_ray_homogeneous_straight,
    lambda orc: bpins.test_maps_linear_gradient_closed_form(orc, 1.0, 2e-6, 5e-5),
    lambda orc: bpins.test_fan_ray_linear_gradient_closed_form_Q(orc, 0.2),
    lambda orc: bpins.test_paraxial_Q_matches_auxiliary_rays(orc, 0, 0.1),
    lambda orc: bpins.test_paraxial_Q_matches_auxiliary_rays(orc, 9, -0.6),
    bpins.test_maps_homogeneous_match_distance,
    bpins.test_maps_match_brute_force_over_all_fan_samples,
    bpins.test_born_dot_product_identity,
    bpins.test_born_point_scatterer_homogeneous,
    bpins.test_born_adjoint_single_datum_homogeneous,
    bpins.test_maps_fermat_against_linking,
    apins.test_zero_alpha_is_lossless,
    apins.test_absorption_uniform_alpha_homogeneous,
    apins.test_absorption_dot_product_identity,
    apins.test_absorption_point_scatterer_homogeneous,
    apins.test_absorption_linear_alpha_brute_force,
]


# reading R13 (an option of the fan-started linking), with its own pins
R13_MUTANTS = {
    "r13_offset_sign": ("    const double a = m1 - p1;\n", "    const double a = p1 - m1;\n"),
    "r13_tilt_dropped": ("        b = ((m2 - p2) - a) / (x2 - x1);", "        b = 0.0 * ((m2 - p2) - a) / (x2 - x1);"),
    "r13_window_off_centre": ("if (fan_points(psi, K, k0 - (n / 2 - 1), n, a_min, step, R, psi_r, tw, mw)) nw = n;",
                              "if (fan_points(psi, K, k0 - n / 2, n, a_min, step, R, psi_r, tw, mw)) nw = n;"),
    "r13_forward_poly_node_dropped": ("if (b != a) l *= (x - t[b]) / (t[a] - t[b]);",
                                      "if (b != a && b != n - 1) l *= (x - t[b]) / (t[a] - t[b]);"),
    "r13_third_angle_through_one_trace": ("r13_angle(tw, mw, nw, prev.theta, prev.m, cur.theta, cur.m, 1, lo, hi)",
                                          "r13_angle(tw, mw, nw, cur.theta, cur.m, 0.0, 0.0, 0, lo, hi)"),
}

R13_PINS = [
    lambda orc: r13pins.test_r13_angle_exact_for_moved_cubic(orc, 1.0, 8),
    lambda orc: r13pins.test_r13_angle_exact_for_moved_cubic(orc, -1.0, 4),
    r13pins.test_r13_angle_linear_window_and_no_sign_change,
    r13pins.test_r13_links_the_same_rays_in_fewer_traces,
]


def _compile_mutant(tmp_path, name, target, old, new):
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, target)).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    shutil.copy(os.path.join(here, "oracle.h"), tmp_path / "oracle.h")
    for f in ("oracle.c", "born.c"):
        text = open(os.path.join(here, f)).read()
        (tmp_path / f).write_text(src.replace(old, new) if f == target else text)
    so = oracle.compile_to(str(tmp_path / f"liboracle_{name}.so"),
                           [str(tmp_path / "oracle.c"), str(tmp_path / "born.c")])
    return oracle.load(so)


def _survives(L, pin_list):
    with oracle.using(L):
        for pin in pin_list:
            try:
                pin(oracle)
            except (AssertionError, ValueError, FloatingPointError):
                return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    L = _compile_mutant(tmp_path, name, "oracle.c", old, new)
    if _survives(L, PINS):
        pytest.fail(f"mutant {name} survived every pin")


@pytest.mark.parametrize("name", sorted(R13_MUTANTS))
def test_r13_mutant_is_caught(name, tmp_path):
    old, new = R13_MUTANTS[name]
    L = _compile_mutant(tmp_path, name, "oracle.c", old, new)
    if _survives(L, R13_PINS):
        pytest.fail(f"mutant {name} survived every R13 pin")


@pytest.mark.parametrize("name", sorted(BSPLINE_MUTANTS))
def test_bspline_mutant_is_caught(name, tmp_path):
    old, new = BSPLINE_MUTANTS[name]
    L = _compile_mutant(tmp_path, name, "oracle.c", old, new)
    if _survives(L, BSPLINE_PINS):
        pytest.fail(f"mutant {name} survived every pin")


BORN_BSPLINE_MUTANTS = {
    "born_bs_second_derivative_basis": ("d2[1] = 3.0 * t - 2.0;", "d2[1] = 3.0 * t - 1.0;"),
    "born_bs_hessian_scale": ("f[F_HXX] = cxx / (h * h);", "f[F_HXX] = cxx / h;"),
    "born_bs_cross_term": ("cxy += dx1[a] * dy1[b] * ak;", "cxy += dx2[a] * by[b] * ak;"),
    "born_bs_gradient_axis": ("cy += bx[a] * dy1[b] * ak;", "cy += dx1[a] * by[b] * ak;"),
    "born_bs_no_prefilter": ("orc_bspline_coef(g, c, F->ac, 0)", "!memcpy(F->ac, c, n * sizeof(double))"),
    "born_heun_end_slope_only": ("for (int q = 0; q < 6; ++q) out[q] = st[q] + 0.5 * hs * (k1[q] + k2[q]);",
                                 "for (int q = 0; q < 6; ++q) out[q] = st[q] + hs * k2[q];"),
}


def _born_in_bspline(pin):
    def run(orc):
        with orc.interpolator("bspline"):
            pin(orc)
    return run


BORN_BSPLINE_PINS = [
    bbpins.test_bspline_fan_ray_homogeneous_straight,
    lambda orc: bbpins.test_bspline_fan_ray_linear_gradient_closed_form_Q(orc, 0.2),
    lambda orc: bbpins.test_bspline_paraxial_Q_matches_auxiliary_rays(orc, 0, 0.1),
    lambda orc: bbpins.test_bspline_paraxial_Q_matches_auxiliary_rays(orc, 40, -0.25),
    bbpins.test_bspline_maps_brute_force,
    bbpins.test_bspline_maps_homogeneous_and_fermat,
    bbpins.test_heun_fan_ray_second_order_Q,
    lambda orc: bbpins.test_heun_paraxial_Q_matches_auxiliary_rays(orc, 0, 0.1),
]
BORN_BSPLINE_PINS = [_born_in_bspline(p) for p in BORN_BSPLINE_PINS]


@pytest.mark.parametrize("name", sorted(BORN_BSPLINE_MUTANTS))
def test_born_bspline_mutant_is_caught(name, tmp_path):
    old, new = BORN_BSPLINE_MUTANTS[name]
    L = _compile_mutant(tmp_path, name, "born.c", old, new)
    if _survives(L, BORN_BSPLINE_PINS):
        pytest.fail(f"mutant {name} survived every pin")


@pytest.mark.parametrize("name", sorted(BORN_MUTANTS))
def test_born_mutant_is_caught(name, tmp_path):
    old, new = BORN_MUTANTS[name]
    L = _compile_mutant(tmp_path, name, "born.c", old, new)
    if _survives(L, BORN_PINS):
        pytest.fail(f"mutant {name} survived every pin")
