"""Plant plausible mistakes in a temporary copy of the oracle and check that
the pins catch every one of them.

Each mutant is compiled from a copy of oracle.c with one textual change (a
dropped term, a flipped sign, a wrong index, a transposed operand, a missing
factor); the committed oracle is never touched. A mutant survives only if all
pins in ``PINS`` still pass, which fails the test.
"""
import os
import shutil

import pytest

import oracle
from tests import test_oracle_pins as pins

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
    "adjoint_missing_chain": ("g_c[j] = -1000.0 * sum / (c_mps[j] * c_mps[j]);",
                              "g_c[j] = -1000.0 * sum / c_mps[j];"),
    "adjoint_drop_alpha": ("gs[S.k[q]] += g_tof[k] * alpha[m] * S.w[q];",
                           "gs[S.k[q]] += g_tof[k] * S.w[q];"),
    "speed_units": ("F->c[k] = v * 1e-3;", "F->c[k] = v * 1e-2;"),
    "slowness_uses_c": ("f[3] += S.w[q] * F->s[S.k[q]];", "f[3] += S.w[q] * F->c[S.k[q]];"),
}

# fast pins first; a mutant is killed by the first pin that fails
PINS = [
    pins.test_bilinear_exact_for_bilinear_field,
    pins.test_homogeneous_straight_rays,
    pins.test_path_matrix_invariants,
    pins.test_adjoint_is_transpose,
    pins.test_hits_land_on_ring_and_within_tol,
    lambda orc: pins.test_linear_gradient_closed_form(orc, 1.0),
    pins.test_rk4_fourth_order_on_circular_arc,
    pins.test_paper_acoustic_length_experiment,
    pins.test_fisheye_ring_closed_form_converges_h2,
    pins.test_adjoint_matches_central_differences,
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    shutil.copy(os.path.join(os.path.dirname(oracle.__file__), "oracle.h"), tmp_path / "oracle.h")
    (tmp_path / "oracle.c").write_text(src.replace(old, new))
    so = oracle.compile_to(str(tmp_path / f"liboracle_{name}.so"), [str(tmp_path / "oracle.c")])
    L = oracle.load(so)
    with oracle.using(L):
        for pin in PINS:
            try:
                pin(oracle)
            except (AssertionError, ValueError, FloatingPointError):
                return
    pytest.fail(f"mutant {name} survived every pin")
