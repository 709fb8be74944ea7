"""Pins of the oracle's cubic B-spline interpolator (arXiv:2511.18511 Sec. 3.3.1,
the second scheme: a C^2 piecewise-cubic field whose control points sit at the
grid nodes, with analytic derivatives; the paper's choice for its Sec. 4
experiments).

Checks that do not come from the oracle: scipy's B-spline routines
(ndimage.spline_filter and map_coordinates of order 3 with the mirror boundary,
which compute the same interpolating spline), the closed-form coefficients of
a cosine mode, the dense inverse of the interpolation matrix written from its
definition, exact reproduction of cubics, C^2 continuity across cell edges,
the derivative against finite differences of the value, the linear-gradient
medium (whose rays are known circles) and the fish-eye lens of Sec. 4.
"""
import json
import os

import numpy as np
import pytest

from paper_2511_18511_gb300 import phantoms as P

from .test_oracle_pins import GOLD, _fisheye_T, _lin_closed_form, _paper_lens_grid

ndimage = pytest.importorskip("scipy.ndimage")


@pytest.fixture
def bs(orc):
    with orc.interpolator("bspline"):
        yield orc


def _interp_matrix(n):
    """(B a)_i = (a_{i-1} + 4 a_i + a_{i+1})/6 with a_{-1} = a_1, a_n = a_{n-2}."""
    B = np.zeros((n, n))
    for i in range(n):
        for k, w in ((i - 1, 1.0), (i, 4.0), (i + 1, 1.0)):
            B[i, abs(k) if k < 0 else (2 * (n - 1) - k if k > n - 1 else k)] += w / 6.0
    return B


def test_bspline_coefficients(bs):
    """Coefficients P^-1 f against scipy's spline_filter (order 3, mirror), the
    cosine closed form a = f / ((4 + 2 cos w)/6) per axis (the mirror extension
    of cos(w i), w = pi m/(n-1), is periodic), and P^-T against the dense
    inverse of the matrix written from its definition."""
    g = P.Grid(30, 25, 0.5)
    f = P.SplitMix64(4).normal(25 * 30).reshape(25, 30)
    a = bs.bspline_coef(g, f)
    np.testing.assert_allclose(a, ndimage.spline_filter(f, order=3, mode="mirror"), atol=1e-13)
    i, j = np.arange(30)[None, :], np.arange(25)[:, None]
    wx, wy = np.pi * 7 / 29, np.pi * 3 / 24
    fc = np.cos(wx * i) * np.cos(wy * j)
    np.testing.assert_allclose(bs.bspline_coef(g, fc), fc * 36.0 / ((4 + 2 * np.cos(wx)) * (4 + 2 * np.cos(wy))),
                               atol=1e-13)
    Pm = np.kron(_interp_matrix(25), _interp_matrix(30))
    np.testing.assert_allclose(bs.bspline_coef(g, f, transpose=True).ravel(), np.linalg.solve(Pm.T, f.ravel()),
                               atol=1e-13)


def test_bspline_samples_match_scipy_everywhere(bs):
    """Off-grid values against scipy's map_coordinates (order 3, mirror,
    prefiltered) over the whole grid, edge cells included; nodal values are
    reproduced exactly; c and s are splined separately."""
    g = P.Grid(30, 25, 0.5)
    c = 1500.0 + 40.0 * P.SplitMix64(6).normal(25 * 30).reshape(25, 30)
    rng = P.SplitMix64(7)
    pts = np.stack([rng.uniform(300, g.x0, g.x0 + 29 * g.h - 1e-9), rng.uniform(300, g.y0, g.y0 + 24 * g.h - 1e-9)], 1)
    f = bs.sample(g, c, pts)
    uv = [(pts[:, 1] - g.y0) / g.h, (pts[:, 0] - g.x0) / g.h]
    np.testing.assert_allclose(f[:, 0], 1e-3 * ndimage.map_coordinates(c, uv, order=3, mode="mirror"), rtol=1e-14)
    np.testing.assert_allclose(f[:, 3], ndimage.map_coordinates(1000.0 / c, uv, order=3, mode="mirror"), rtol=1e-14)
    x, y = g.node_xy()
    f = bs.sample(g, c, np.stack([x.ravel(), y.ravel()], 1))
    np.testing.assert_allclose(f[:, 0], 1e-3 * c.ravel(), rtol=1e-14)


# a bicubic c (m/s) with every monomial x^p y^q, p, q <= 3
COEF = {(0, 0): 1500.0, (1, 0): 2.0, (0, 1): -1.5, (2, 0): 0.02, (1, 1): 0.03, (0, 2): -0.025,
        (3, 0): 4e-4, (2, 1): -3e-4, (1, 2): 2e-4, (0, 3): 5e-4, (3, 3): 1e-7, (2, 2): -2e-6}


def test_bspline_reproduces_cubics_with_exact_gradient(bs):
    """A bicubic is itself a C^2 cubic spline, so the interpolating spline
    reproduces it, with its gradient, away from the mirrored edges (whose
    influence decays as (2 - sqrt 3)^k over k cells)."""
    g = P.Grid(80, 80, 0.25)
    x, y = g.node_xy()
    c = sum(a * x ** p * y ** q for (p, q), a in COEF.items())
    rng = P.SplitMix64(21)
    pts = np.stack([rng.uniform(300, -4.0, 4.0), rng.uniform(300, -4.0, 4.0)], 1)   # >= 24 cells inside
    X, Y = pts[:, 0], pts[:, 1]
    f = bs.sample(g, c, pts)
    val = sum(a * X ** p * Y ** q for (p, q), a in COEF.items())
    ddx = sum(a * p * X ** max(p - 1, 0) * Y ** q for (p, q), a in COEF.items())
    ddy = sum(a * q * X ** p * Y ** max(q - 1, 0) for (p, q), a in COEF.items())
    np.testing.assert_allclose(f[:, 0], 1e-3 * val, rtol=1e-13)
    np.testing.assert_allclose(f[:, 1], 1e-3 * ddx, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(f[:, 2], 1e-3 * ddy, rtol=1e-9, atol=1e-14)


def test_bspline_is_c2_across_cell_edges(bs):
    """Value, gradient and (one-sided finite differences of the gradient) second
    derivatives agree on both sides of node lines for a rough random field;
    bilinear sampling is only C^0 there."""
    g = P.Grid(32, 32, 0.5)
    c = 1500.0 + 40.0 * P.SplitMix64(5).normal(32 * 32).reshape(32, 32)
    eps = 1e-6 * g.h
    for k, (i, yv) in enumerate([(9, 0.37), (14, -2.11), (20, 1.5)]):
        xn = g.x0 + i * g.h
        a = bs.sample(g, c, np.array([[xn - eps, yv], [xn + eps, yv]]))
        assert abs(a[0, 0] - a[1, 0]) < 1e-6 * abs(a[0, 0])
        assert abs(a[0, 1] - a[1, 1]) < 1e-4 * np.abs(a[:, 1]).max()
        l = bs.sample(g, c, np.array([[xn - 2 * eps, yv], [xn - eps, yv]]))
        r = bs.sample(g, c, np.array([[xn + eps, yv], [xn + 2 * eps, yv]]))
        dl, dr = (l[1, 1] - l[0, 1]) / eps, (r[1, 1] - r[0, 1]) / eps
        assert abs(dl - dr) < 1e-3 * max(abs(dl), 1e-6), (k, dl, dr)
        yn = g.y0 + (i + 1) * g.h
        l = bs.sample(g, c, np.array([[yv, yn - 2 * eps], [yv, yn - eps]]))
        r = bs.sample(g, c, np.array([[yv, yn + eps], [yv, yn + 2 * eps]]))
        dl, dr = (l[1, 2] - l[0, 2]) / eps, (r[1, 2] - r[0, 2]) / eps
        assert abs(dl - dr) < 1e-3 * max(abs(dl), 1e-6), (k, dl, dr)


def test_bspline_gradient_is_the_derivative_of_the_value(bs):
    """The analytic gradient equals central differences of the sampled value."""
    g = P.Grid(40, 40, 0.5)
    c = 1500.0 + 30.0 * P.SplitMix64(9).normal(1600).reshape(40, 40)
    rng = P.SplitMix64(33)
    pts = np.stack([rng.uniform(50, -8.0, 8.0), rng.uniform(50, -8.0, 8.0)], 1)
    e = 1e-4 * g.h
    f = bs.sample(g, c, pts)
    fx = (bs.sample(g, c, pts + [e, 0])[:, 0] - bs.sample(g, c, pts - [e, 0])[:, 0]) / (2 * e)
    fy = (bs.sample(g, c, pts + [0, e])[:, 0] - bs.sample(g, c, pts - [0, e])[:, 0]) / (2 * e)
    scale = np.abs(f[:, 1:3]).max()
    assert np.abs(f[:, 1] - fx).max() < 1e-6 * scale
    assert np.abs(f[:, 2] - fy).max() < 1e-6 * scale


def test_bspline_homogeneous_straight_rays(bs):
    """A constant field is its own spline: T = chord / c, rows sum to the chord."""
    g, tx, R = P.Grid(128, 128, 0.5), P.ring(24, 30.0), 30.0
    c = P.homogeneous(g, 1500.0)
    pairs = P.all_pairs(24)
    r = bs.link(g, c, tx, R, 0.05)
    chord = np.linalg.norm(tx[pairs[:, 0]] - tx[pairs[:, 1]], axis=1)
    np.testing.assert_allclose(r["tof"], chord / 1.5, rtol=1e-12)
    assert (r["iters"] == 1).all()
    rp, col, val = bs.path_matrix(g, c, tx, R, 0.05, r["theta"])
    np.testing.assert_allclose(np.add.reduceat(val, rp[:-1]), chord, rtol=1e-12)


@pytest.mark.parametrize("gslope", [1.0, 3.0])
def test_bspline_linear_gradient_closed_form(bs, gslope):
    """c = c_m + g y is reproduced exactly with its gradient (far from the grid
    edges), so rays are the analytic circles, and the spline of s = 1/c is
    O(h^4) accurate: T and the launch angles match the closed forms to the RK4
    and linking residuals (measured 2e-10 and 1.7e-9 relative)."""
    g, tx, R = P.Grid(200, 200, 0.5), P.ring(64, 30.0), 30.0
    c = P.linear_gradient(g, 1500.0, gslope)
    pairs = P.all_pairs(64)
    r = bs.link(g, c, tx, R, 0.05, tol=1e-9)
    assert (r["status"] == 0).all() and r["iters"].max() <= 6
    rel = r["tof"] / _lin_closed_form(tx, pairs, 1500.0, gslope) - 1
    assert np.abs(rel).max() < 5e-9 * gslope ** 2
    xe, xr = tx[pairs[:, 0]], tx[pairs[:, 1]]
    yc = -1500.0 / gslope
    dx = xe[:, 0] - xr[:, 0]
    ok = np.abs(dx) > 1e-6
    xc = ((xe[:, 0] ** 2 - xr[:, 0] ** 2) + (xe[:, 1] - yc) ** 2 - (xr[:, 1] - yc) ** 2) / (2 * np.where(ok, dx, 1))
    t = np.stack([-(xe[:, 1] - yc), xe[:, 0] - xc], 1)
    t *= np.sign((t * (xr - xe)).sum(1))[:, None]
    th = np.arctan2(t[:, 1], t[:, 0])
    assert np.abs(np.angle(np.exp(1j * (th - r["theta"]))))[ok].max() < 1e-9


def test_bspline_path_matrix_and_adjoint(bs):
    """The rows weight the slowness coefficients: T = L P^-1 s exactly, and the
    adjoint is -(1000/c^2) P^-T L^T g (P^-T from the dense definition)."""
    w = P.cfg_small(n_tx=16)
    r = bs.link(w.grid, w.c, w.tx, w.ring_radius, w.ds)
    assert (r["status"] == 0).all()
    rp, col, val = bs.path_matrix(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"])
    a_s = bs.bspline_coef(w.grid, 1000.0 / w.c).ravel()
    np.testing.assert_allclose(np.add.reduceat(val * a_s[col], rp[:-1]), r["tof"], rtol=1e-12)
    gt = P.SplitMix64(3).normal(len(r["tof"]))
    LTg = np.zeros(a_s.size)
    np.add.at(LTg, col, val * gt[np.repeat(np.arange(len(gt)), np.diff(rp))])
    Pm = np.kron(_interp_matrix(w.grid.ny), _interp_matrix(w.grid.nx))
    ref = -1000.0 * np.linalg.solve(Pm.T, LTg) / w.c.ravel() ** 2
    gc = bs.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"], gt).ravel()
    assert np.abs(gc - ref).max() <= 1e-11 * np.abs(ref).max()


def test_bspline_fisheye_ring_closed_form(bs):
    """The Maxwell fish-eye ring of Sec. 4 with the spline: linked travel times
    reach the great-circle closed form ~400x closer than with bilinear sampling
    (measured 5.5e-8 vs 2.1e-5 RMS relative at h = 0.8), and the residual, now
    the O(ds^2) trapezoid rule at ds = h/10, falls ~4x when h halves."""
    pairs = P.all_pairs(24)
    errs = []
    for n, h, ds in ((128, 0.8, 0.08), (256, 0.4, 0.04)):
        w = P.cfg_fisheye(n=n, n_tx=24, h=h, ds=ds)
        r = bs.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-6)
        assert (r["status"] == 0).all()
        rel = r["tof"] / _fisheye_T(w.tx, pairs) - 1
        errs.append(np.sqrt(np.mean(rel ** 2)))
    assert errs[0] < 2e-7
    assert 3.0 < errs[0] / errs[1] < 5.5, errs


def _length_experiment():
    gold = json.load(open(os.path.join(GOLD, "fisheye_paper.json")))
    ex = gold["length_experiment"]
    xp, xq = np.array(ex["x_p"]), np.array(ex["x_intercept"])
    axis = np.arctan2(*(np.array(ex["x_c"]) - xp)[::-1])
    thetas = axis + np.linspace(ex["theta_min"], ex["theta_max"], ex["n_rays"])
    return gold, ex, xp, xq, thetas


def test_bspline_paper_acoustic_length_experiment(bs):
    """Sec. 4.2 in the paper's own set-up (B-spline interpolation, dx = 2 pi a/360,
    101 rays from [0, a] to [0, -a], L_true = a pi/2): the mean relative error
    RE_al is set by the ray step, not the grid: it falls ~4x when ds/dx halves
    on the paper's grid, and ~4x when grid and step are both refined 2x."""
    gold, ex, xp, xq, thetas = _length_experiment()
    re = {}
    for refine, ratio in ((1, 1.0), (1, 0.5), (2, 1.0)):
        h = gold["dx_over_a"] * gold["a"] / refine
        g, c = _paper_lens_grid(h, 1.15)
        L = np.array([bs.trace(g, c, 1.0, xp, xq, th, ratio * h, record=False)["T"] for th in thetas])
        re[refine, ratio] = np.mean((L - ex["L_true"]) / ex["L_true"]) * 100
    assert abs(re[1, 1.0]) < 3e-3
    assert 3.5 < re[1, 1.0] / re[1, 0.5] < 4.5 and 3.5 < re[1, 1.0] / re[2, 1.0] < 4.5, re


def test_bspline_paper_radius_experiment(bs):
    """Sec. 4.1: the ray from [0, a] launched normal to [a, 0] - [0, a] circles
    [a, 0] with radius sqrt(2) a; with the spline's analytic gradient the mean
    radius deviation RE_rd on the paper's grid is far below the bilinear one
    (measured 3.7e-6 % against 5.1e-3 %)."""
    gold = json.load(open(os.path.join(GOLD, "fisheye_paper.json")))
    ex = gold["radius_experiment"]
    xp, xc = np.array(ex["x_p"]), np.array(ex["x_c"])
    ax = xc - xp
    d0 = np.array([ax[1], -ax[0]]) / np.linalg.norm(ax)
    th = np.arctan2(d0[1], d0[0])
    h = gold["dx_over_a"]
    g, c = _paper_lens_grid(h, 2.6)
    n = int(np.ceil(2 * np.pi * ex["R_true"] / h * 1.2))
    pts = bs.march(g, c, xp[0], xp[1], th, h, n)
    dist = np.linalg.norm(pts - xp, axis=1)
    half = len(pts) // 2
    stop = half + int(np.argmin(dist[half:]))
    assert dist[stop] < h
    dev = np.abs(np.linalg.norm(pts[1:stop + 1] - xc, axis=1) - ex["R_true"]) / ex["R_true"]
    assert dev.mean() * 100 < 2e-5
