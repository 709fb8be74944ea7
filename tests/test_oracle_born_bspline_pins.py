"""Pins of the ray-Born oracle with the cubic B-spline sampler (paper Sec.
3.3.1: the toolbox uses the spline for ray-Born because its analytic first and
second derivatives are essential for the ray and amplitude computations).

The decisive check is the paper's auxiliary-ray Jacobian (Sec. 3.5): with the
spline, the Hessian that drives the paraxial ray is the exact derivative of
the gradient that drives the rays, so the paraxial Q equals the separation of
two neighbouring rays to ~1e-9 (bilinear sampling with central-difference
Hessians leaves ~1e-3). Also: straight rays in a constant medium, the
closed-form Q of the linear-gradient medium, the map rule recomputed by brute
force from recorded samples, and Fermat against the separately pinned
linking oracle (with the same sampler).
"""
import numpy as np
import pytest

from paper_2511_18511_gb300 import phantoms as P

from . import test_oracle_born_pins as B
from .test_oracle_born_pins import C0, _homog


@pytest.fixture
def bs(orc):
    with orc.interpolator("bspline"):
        yield orc


def test_bspline_fan_ray_homogeneous_straight(bs):
    """A constant field is its own spline (to the prefilter's rounding): the ray
    is straight, Q the distance, P = 1/c, T = distance / c."""
    g, c, tx, R = _homog()
    r = bs.fan_ray(g, c, R, tx[0], np.pi + 0.3, 0.05)
    dist = np.hypot(r["x"] - tx[0, 0], r["y"] - tx[0, 1])
    assert len(dist) > 100
    np.testing.assert_allclose(r["Q"], dist, atol=1e-10)
    np.testing.assert_allclose(r["P"], 1.0 / C0, rtol=1e-12)
    np.testing.assert_allclose(r["T"], dist / C0, atol=1e-11)


@pytest.mark.parametrize("theta_off", [0.2, -0.5, 0.8])
def test_bspline_fan_ray_linear_gradient_closed_form_Q(bs, theta_off):
    """c = c_m + g y is reproduced by the spline with a zero Hessian, so
    P = 1/c_t and Q = |x - x_e| / |cos a| along the circular ray. The grid
    reaches 19 cells beyond the ring: the mirror extension of a linear field
    kinks at the grid edge, and that kink's curvature decays only as
    (2 - sqrt 3)^k over k cells (at 3.5 cells it moves P by 4e-10)."""
    g = P.Grid(160, 160, 0.5)
    c = P.linear_gradient(g)
    tx = P.ring(16, 30.0)
    th = np.pi + theta_off
    r = bs.fan_ray(g, c, 30.0, tx[0], th, 0.05)
    q = np.abs(r["x"] - tx[0, 0]) / abs(np.cos(th))
    np.testing.assert_allclose(r["Q"][1:], q[1:], rtol=1e-9)
    c_t = 1e-3 * (1500.0 + tx[0, 1])
    np.testing.assert_allclose(r["P"], 1.0 / c_t, rtol=1e-11)


@pytest.mark.parametrize("k,off", [(0, 0.1), (9, -0.6), (18, 0.9), (40, -0.25)])
def test_bspline_paraxial_Q_matches_auxiliary_rays(bs, k, off):
    """Paraxial Q against the normal separation of rays launched at theta +-
    1e-6 over the whole ray, broad Gaussian inclusions: measured <= 1.8e-9
    relative with the spline (9.6e-4 bilinear)."""
    w = P.cfg_born_small()
    e = w.tx[k]
    th = np.arctan2(e[1], e[0]) + np.pi + off
    d = 1e-6
    a = bs.fan_ray(w.grid, w.c, w.ring_radius, e, th, w.ds)
    p = bs.fan_ray(w.grid, w.c, w.ring_radius, e, th + d, w.ds)
    m = bs.fan_ray(w.grid, w.c, w.ring_radius, e, th - d, w.ds)
    n = min(len(a["x"]), len(p["x"]), len(m["x"]))
    q = (-a["dy"][:n] * (p["x"][:n] - m["x"][:n]) + a["dx"][:n] * (p["y"][:n] - m["y"][:n])) / (2 * d)
    assert n > 200
    err = np.abs(a["Q"][1:n] - q[1:n]).max() / np.abs(q[1:n]).max()
    assert err < 2e-8, err


def test_bspline_maps_brute_force(bs):
    """The map rule recomputed from the recorded samples of every fan ray."""
    B.test_maps_match_brute_force_over_all_fan_samples(bs)


def test_bspline_maps_homogeneous_and_fermat(bs):
    """Homogeneous maps match the distance; first-arrival maps meet the linked
    travel times of the linking oracle (Fermat) with the spline on both."""
    B.test_maps_homogeneous_match_distance(bs)
    B.test_maps_fermat_against_linking(bs)


# ---------------------------------------------------------------- Heun's RK2 (the paper's default)

def test_heun_fan_ray_second_order_Q(orc):
    """With Heun's RK2 the paraxial Q along the circular ray of the linear-
    gradient medium (closed form |x - x_e| / |cos a|) converges at second
    order: the error falls 4x per halving of ds (RK4: 16x)."""
    g = P.Grid(160, 160, 0.5)
    c = P.linear_gradient(g, 1500.0, 20.0)
    tx = P.ring(16, 30.0)
    th = np.pi + 0.5
    errs = []
    with orc.integrator("heun"):
        for ds in (0.4, 0.2, 0.1):
            r = orc.fan_ray(g, c, 30.0, tx[0], th, ds)
            q = np.abs(r["x"] - tx[0, 0]) / abs(np.cos(th))
            errs.append(np.abs(r["Q"][1:] / q[1:] - 1).max())
    assert errs[0] < 5e-6
    assert all(3.5 < errs[i] / errs[i + 1] < 4.5 for i in range(2)), errs


@pytest.mark.parametrize("k,off", [(0, 0.1), (9, -0.6)])
def test_heun_paraxial_Q_matches_auxiliary_rays(bs, k, off):
    """A Runge-Kutta step of the paraxial pair is the derivative of the same
    step of the ray, so the auxiliary-ray Jacobian and Q agree with Heun too
    (measured <= 6e-8 with the spline)."""
    w = P.cfg_born_small()
    e = w.tx[k]
    th = np.arctan2(e[1], e[0]) + np.pi + off
    d = 1e-6
    with bs.integrator("heun"):
        a = bs.fan_ray(w.grid, w.c, w.ring_radius, e, th, w.ds)
        p = bs.fan_ray(w.grid, w.c, w.ring_radius, e, th + d, w.ds)
        m = bs.fan_ray(w.grid, w.c, w.ring_radius, e, th - d, w.ds)
    n = min(len(a["x"]), len(p["x"]), len(m["x"]))
    q = (-a["dy"][:n] * (p["x"][:n] - m["x"][:n]) + a["dx"][:n] * (p["y"][:n] - m["y"][:n])) / (2 * d)
    err = np.abs(a["Q"][1:n] - q[1:n]).max() / np.abs(q[1:n]).max()
    assert err < 3e-7, err
