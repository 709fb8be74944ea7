"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test checks the oracle against something other than itself: an exact
solution of the ray equations, a textbook identity, a brute-force search, or
the paper's own analytic fish-eye experiments (arXiv:2511.18511, Sec. 4).
The mutation tests (test_oracle_mutations.py) show that plausible mistakes in
the oracle fail at least one of these.
"""
import json
import os

import numpy as np
import pytest

from paper_2511_18511_gb300 import phantoms as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _small_ring(n_tx=64):
    g = P.Grid(128, 128, 0.5)
    return g, P.ring(n_tx, 30.0), 30.0


# ---------------------------------------------------------------- interpolation

def test_bilinear_exact_for_bilinear_field(orc):
    """Bilinear interpolation reproduces a bilinear c exactly (Sec. 3.3.1); the
    central-difference gradient of a quadratic is exact inside the grid and
    linear, hence also interpolated exactly."""
    g = P.Grid(40, 30, 0.7)
    x, y = g.node_xy()
    c_lin = 1500.0 + 3.0 * x - 2.0 * y + 0.05 * x * y
    rng = P.SplitMix64(11)
    pts = np.stack([rng.uniform(200, g.x0 + g.h, -g.x0 - g.h),
                    rng.uniform(200, g.y0 + g.h, -g.y0 - g.h)], 1)
    f = orc.sample(g, c_lin, pts)
    X, Y = pts[:, 0], pts[:, 1]
    np.testing.assert_allclose(f[:, 0], 1e-3 * (1500.0 + 3.0 * X - 2.0 * Y + 0.05 * X * Y), rtol=1e-13)
    c_q = 1500.0 + 2.0 * x + 0.01 * x * x - 0.03 * y * y + 0.02 * x * y
    f = orc.sample(g, c_q, pts)
    np.testing.assert_allclose(f[:, 1], 1e-3 * (2.0 + 0.02 * X + 0.02 * Y), rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(f[:, 2], 1e-3 * (-0.06 * Y + 0.02 * X), rtol=1e-11, atol=1e-15)
    # one-sided differences at the four edges; for the quadratic the forward
    # difference at x is c'(x) + c''(x) h/2 and the backward one c'(x) - c''(x) h/2
    c, gx, gy, s = orc.field(g, c_q)
    xs, ys = x[0, :], y[:, 0]
    h = g.h
    np.testing.assert_allclose(gx[:, 0], 1e-3 * (2.0 + 0.02 * xs[0] + 0.01 * h + 0.02 * ys), rtol=1e-11)
    np.testing.assert_allclose(gx[:, -1], 1e-3 * (2.0 + 0.02 * xs[-1] - 0.01 * h + 0.02 * ys), rtol=1e-11)
    np.testing.assert_allclose(gy[0, :], 1e-3 * (-0.06 * ys[0] - 0.03 * h + 0.02 * xs), rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(gy[-1, :], 1e-3 * (-0.06 * ys[-1] + 0.03 * h + 0.02 * xs), rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(s * c, 1.0, rtol=1e-15)


# ---------------------------------------------------------------- straight rays

def test_homogeneous_straight_rays(orc):
    """c = const: rays are straight, T = |x_r - x_e|/c, the straight start is
    already linked (one trace), and every system-matrix row sums to the chord."""
    g, tx, R = _small_ring(32)
    c = P.homogeneous(g, 1500.0)
    pairs = P.all_pairs(32)
    r = orc.link(g, c, tx, R, 0.05)
    chord = np.linalg.norm(tx[pairs[:, 0]] - tx[pairs[:, 1]], axis=1)
    np.testing.assert_allclose(r["tof"], chord / 1.5, rtol=1e-12)
    assert (r["iters"] == 1).all() and (r["status"] == 0).all()
    straight = np.arctan2(*(tx[pairs[:, 1]] - tx[pairs[:, 0]])[:, ::-1].T)
    assert np.abs(np.angle(np.exp(1j * (r["theta"] - straight)))).max() < 1e-14
    np.testing.assert_allclose(r["hit"], tx[pairs[:, 1]], atol=1e-9)
    rp, col, val = orc.path_matrix(g, c, tx, R, 0.05, r["theta"])
    rows = np.add.reduceat(val, rp[:-1])
    np.testing.assert_allclose(rows, chord, rtol=1e-12)


# ---------------------------------------------------------------- linear gradient

def _lin_closed_form(tx, pairs, c_mid, gslope):
    xe, xr = tx[pairs[:, 0]], tx[pairs[:, 1]]
    gm = gslope * 1e-3
    ce = 1e-3 * c_mid + gm * xe[:, 1]
    cr = 1e-3 * c_mid + gm * xr[:, 1]
    D = np.linalg.norm(xe - xr, axis=1)
    return np.arccosh(1.0 + gm * gm * D * D / (2.0 * ce * cr)) / gm


@pytest.mark.parametrize("gslope", [1.0, 3.0])
def test_linear_gradient_closed_form(orc, gslope):
    """c = c_m + g*y: rays are circular arcs centred on the line c = 0 and
    T = arccosh(1 + g^2 |dx|^2 / (2 c_e c_r)) / g. Bilinear interpolation and
    central differences are exact for a linear c, so the residual is RK4 plus
    the interpolated slowness, about h^2 g^2/(4 c^2) relative."""
    g, tx, R = _small_ring(64)
    c = P.linear_gradient(g, 1500.0, gslope)
    pairs = P.all_pairs(64)
    r = orc.link(g, c, tx, R, 0.05, tol=1e-9)
    assert (r["status"] == 0).all()
    # smooth monotone misfit: the secant converges superlinearly (measured <= 6
    # traces at tol 1e-9, the orientation probe included)
    assert r["iters"].max() <= 6
    T = _lin_closed_form(tx, pairs, 1500.0, gslope)
    bound = 1.5 * (g.h * gslope * 1e-3) ** 2 / (4 * 1.47 ** 2)
    assert np.abs(r["tof"] / T - 1).max() < bound
    # launch angle = tangent of the analytic circle at the emitter
    xe, xr = tx[pairs[:, 0]], tx[pairs[:, 1]]
    yc = -1500.0 / gslope
    dx = xe[:, 0] - xr[:, 0]
    ok = np.abs(dx) > 1e-6
    xc = ((xe[:, 0] ** 2 - xr[:, 0] ** 2) + (xe[:, 1] - yc) ** 2 - (xr[:, 1] - yc) ** 2) / (2 * np.where(ok, dx, 1))
    t = np.stack([-(xe[:, 1] - yc), xe[:, 0] - xc], 1)
    t *= np.sign((t * (xr - xe)).sum(1))[:, None]
    th = np.arctan2(t[:, 1], t[:, 0])
    assert np.abs(np.angle(np.exp(1j * (th - r["theta"]))))[ok].max() < 1e-9


def test_rk4_fourth_order_on_circular_arc(orc):
    """In c = c_m + g*y the ray through p with direction d is the circle centred
    where the normal at p meets y = -c_m/g. The deviation of the marched points
    from that circle must shrink ~16x when ds halves (classic RK4)."""
    g = P.Grid(128, 128, 0.5)
    c = P.linear_gradient(g, 1500.0, 20.0)
    p = np.array([-20.0, 0.0])
    th = 0.3
    d = np.array([np.cos(th), np.sin(th)])
    yc = -1500.0 / 20.0
    t = (yc - p[1]) / d[0]
    centre = np.array([p[0] - t * d[1], yc])
    errs = []
    for ds in (2.0, 1.0, 0.5):
        n = int(round(36.0 / ds))
        pts = orc.march(g, c, p[0], p[1], th, ds, n)
        errs.append(np.abs(np.linalg.norm(pts - centre, axis=1) - abs(t)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 11.0 < r1 < 22.0 and 11.0 < r2 < 22.0, errs


def _arc_errors(orc, steps):
    g = P.Grid(128, 128, 0.5)
    c = P.linear_gradient(g, 1500.0, 20.0)
    p = np.array([-20.0, 0.0])
    th = 0.3
    d = np.array([np.cos(th), np.sin(th)])
    yc = -1500.0 / 20.0
    t = (yc - p[1]) / d[0]
    centre = np.array([p[0] - t * d[1], yc])
    errs = []
    for ds in steps:
        n = int(round(36.0 / ds))
        pts = orc.march(g, c, p[0], p[1], th, ds, n)
        errs.append(np.abs(np.linalg.norm(pts - centre, axis=1) - abs(t)).max())
    return errs


def test_heun_second_order_on_circular_arc(orc):
    """The paper's default integrator (Sec. 3.2.3, Heun's second-order
    Runge-Kutta): on the same exact circular arc the deviation shrinks ~4x per
    halving of ds; straight rays stay exact."""
    with orc.integrator("heun"):
        errs = _arc_errors(orc, (1.0, 0.5, 0.25))
        g = P.Grid(64, 64, 0.5)
        pts = orc.march(g, P.homogeneous(g), -10.0, 3.0, 0.7, 0.3, 40)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs
    s = np.arange(41) * 0.3
    np.testing.assert_allclose(pts, np.stack([-10.0 + s * np.cos(0.7), 3.0 + s * np.sin(0.7)], 1), atol=1e-12)


def test_heun_linking_converges_to_analytic_circles(orc):
    """Heun linking in c = c_m + g y (g = 5 (m/s)/mm): the linked launch angles
    approach the tangents of the analytic circles at second order in ds (ratio
    ~4 per halving; RK4 reaches them to 1e-13 at any of these steps)."""
    g, tx, R = _small_ring(16)
    gs = 5.0
    c = P.linear_gradient(g, 1500.0, gs)
    pairs = np.array([[0, 5], [3, 11], [8, 14], [2, 9]], np.int32)
    xe, xr = tx[pairs[:, 0]], tx[pairs[:, 1]]
    yc = -1500.0 / gs
    dx = xe[:, 0] - xr[:, 0]
    xc = ((xe[:, 0] ** 2 - xr[:, 0] ** 2) + (xe[:, 1] - yc) ** 2 - (xr[:, 1] - yc) ** 2) / (2 * dx)
    t = np.stack([-(xe[:, 1] - yc), xe[:, 0] - xc], 1)
    t *= np.sign((t * (xr - xe)).sum(1))[:, None]
    th = np.arctan2(t[:, 1], t[:, 0])
    errs = []
    with orc.integrator("heun"):
        for ds in (0.4, 0.2, 0.1):
            r = orc.link(g, c, tx, R, ds, tol=1e-10, pairs=pairs)
            assert (r["status"] == 0).all()
            errs.append(np.abs(np.angle(np.exp(1j * (th - r["theta"])))).max())
    assert all(3.6 < errs[k] / errs[k + 1] < 4.4 for k in range(2)), errs


# ---------------------------------------------------------------- fish-eye lens

def _fisheye_T(tx, pairs, a=40.0, c0=1.5):
    xe, xr = tx[pairs[:, 0]], tx[pairs[:, 1]]
    chord = a * np.linalg.norm(xe - xr, axis=1) / np.sqrt((a * a + (xe ** 2).sum(1)) * (a * a + (xr ** 2).sum(1)))
    sigma = 2.0 * np.arcsin(chord)
    # inside a ring of radius > a the ray runs the major arc of the great circle
    return a * (2.0 * np.pi - sigma) / c0


def test_fisheye_ring_closed_form_converges_h2(orc):
    """Maxwell fish-eye c = c0 (1 + r^2/a^2)/2 (Sec. 4): the optical metric is a
    sphere of radius a, so T = a (2 pi - sigma)/c0 with sigma the great-circle
    angle; linked rays must reach it with an O(h^2) interpolation error."""
    pairs = P.all_pairs(24)
    errs = []
    for n, h, ds in ((128, 0.8, 0.08), (256, 0.4, 0.04)):
        w = P.cfg_fisheye(n=n, n_tx=24, h=h, ds=ds)
        r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-6)
        assert (r["status"] == 0).all()
        rel = r["tof"] / _fisheye_T(w.tx, pairs) - 1
        errs.append(np.sqrt(np.mean(rel ** 2)))
    assert errs[1] < 3e-5
    assert 3.0 < errs[0] / errs[1] < 5.5, errs


def test_fisheye_rays_follow_circles(orc):
    """Every fish-eye ray from e passes through the conjugate point
    -(a^2/|e|^2) e (Sec. 4), so the linked ray e->r lies on the circle through
    e, the conjugate point and r."""
    w = P.cfg_fisheye(n=256, n_tx=16, h=0.4, ds=0.04)
    pairs = P.all_pairs(16)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-6)
    worst = 0.0
    for k in range(0, len(pairs), 7):
        e, q = pairs[k]
        xe, xr = w.tx[e], w.tx[q]
        xc = -(40.0 ** 2 / (xe @ xe)) * xe
        A = np.array([[2 * (xr - xe)[0], 2 * (xr - xe)[1]], [2 * (xc - xe)[0], 2 * (xc - xe)[1]]])
        b = np.array([xr @ xr - xe @ xe, xc @ xc - xe @ xe])
        ctr = np.linalg.solve(A, b)
        rad = np.linalg.norm(xe - ctr)
        tr = orc.trace(w.grid, w.c, w.ring_radius, xe, xr, r["theta"][k], w.ds)
        dev = np.abs(np.linalg.norm(tr["pts"] - ctr, axis=1) / rad - 1).max()
        worst = max(worst, dev)
    assert worst < 2e-4, worst


def _paper_lens_grid(h, extent):
    n = 2 * int(np.ceil(extent / h)) + 1
    g = P.Grid(n, n, h)
    x, y = g.node_xy()
    # n = n(x_o)/(1 + r^2/a^2) with n(x_o) = a = 1; c = 1/n in mm/us -> 1000/n m/s
    return g, 1000.0 * (1.0 + x * x + y * y)


def test_paper_acoustic_length_experiment(orc):
    """Sec. 4.2, 2D: 101 rays from [0, a] at angles in [-pi/3, pi/3] about the
    axis to [0, 0] all reach [0, -a] with acoustic length L_true = a pi/2.
    On the paper's grid (dx = 2 pi a/360) at ds/dx = 1 the deviation must be
    small and shrink ~4x when the grid is refined 2x (interpolation-dominated,
    as the paper observes for small ds/dx)."""
    gold = json.load(open(os.path.join(GOLD, "fisheye_paper.json")))
    ex = gold["length_experiment"]
    xp, xq = np.array(ex["x_p"]), np.array(ex["x_intercept"])
    axis = np.arctan2(*(np.array(ex["x_c"]) - xp)[::-1])
    thetas = axis + np.linspace(ex["theta_min"], ex["theta_max"], ex["n_rays"])
    re = []
    for refine in (1, 2):
        h = gold["dx_over_a"] * gold["a"] / refine
        g, c = _paper_lens_grid(h, 1.15)
        L, hits = [], []
        for th in thetas:
            t = orc.trace(g, c, 1.0, xp, xq, th, h, record=False)
            L.append(t["T"])
            hits.append(t["hit"])
        L = np.array(L)
        assert np.abs(np.array(hits) - xq).max() < 3e-4 / refine ** 2
        re.append(np.mean((L - ex["L_true"]) / ex["L_true"]) * 100)
    assert abs(re[0]) < 1e-2 and 3.0 < re[0] / re[1] < 5.0, re


def test_paper_radius_experiment(orc):
    """Sec. 4.1, 2D: the ray from [0, a] launched clockwise normal to [a, 0] - [0, a]
    circles [a, 0] with radius sqrt(2) a and returns to its start. Mean radius
    deviation RE_rd over the loop must be small and shrink with the grid."""
    gold = json.load(open(os.path.join(GOLD, "fisheye_paper.json")))
    ex = gold["radius_experiment"]
    xp, xc = np.array(ex["x_p"]), np.array(ex["x_c"])
    ax = xc - xp
    d0 = np.array([ax[1], -ax[0]]) / np.linalg.norm(ax)   # clockwise about x_c
    th = np.arctan2(d0[1], d0[0])
    out = []
    for refine in (1, 2):
        h = gold["dx_over_a"] / refine
        g, c = _paper_lens_grid(h, 2.6)
        ds = h
        n = int(np.ceil(2 * np.pi * ex["R_true"] / ds * 1.2))
        pts = orc.march(g, c, xp[0], xp[1], th, ds, n)
        dist = np.linalg.norm(pts - xp, axis=1)
        # p*: the last point before the loop closes, within ds of the start
        half = len(pts) // 2
        stop = half + int(np.argmin(dist[half:]))
        assert dist[stop] < ds
        dev = np.abs(np.linalg.norm(pts[1:stop + 1] - xc, axis=1) - ex["R_true"]) / ex["R_true"]
        out.append(dev.mean() * 100)
    assert out[0] < 0.05 and out[1] < out[0] / 2.5, out


# ---------------------------------------------------------------- reciprocity

def test_reciprocity(orc):
    """T(e -> r) = T(r -> e) (Fermat): the discrete rays traced from opposite ends
    agree to the integration error."""
    w = P.cfg_small(n_tx=32)
    pairs = P.all_pairs(32)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-9)
    M = np.zeros((32, 32))
    M[pairs[:, 0], pairs[:, 1]] = r["tof"]
    assert np.abs(M - M.T).max() / M.max() < 2e-7


# ---------------------------------------------------------------- system matrix and adjoint

def test_path_matrix_invariants(orc):
    """T = L s exactly; rows sum to the ray length ((M-1) ds + ds') plus the
    endpoint weight; entries of L are non-negative up to that weight."""
    w = P.cfg_small(n_tx=24)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds)
    rp, col, val = orc.path_matrix(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"])
    _, _, _, s = orc.field(w.grid, w.c)
    sf = s.ravel()
    T_L = np.add.reduceat(val * sf[col], rp[:-1])
    np.testing.assert_allclose(T_L, r["tof"], rtol=1e-12)
    pairs = P.all_pairs(24)
    for k in (0, 100, 333, len(pairs) - 1):
        e, q = pairs[k]
        tr = orc.trace(w.grid, w.c, w.ring_radius, w.tx[e], w.tx[q], r["theta"][k], w.ds)
        length = (tr["n_pts"] - 2) * w.ds + tr["dsp"]
        corr = tr["dir"] @ (w.tx[q] - tr["hit"])
        np.testing.assert_allclose(val[rp[k]:rp[k + 1]].sum(), length + corr, rtol=1e-12)
        assert abs(corr) < 1e-4
    assert val.min() > -1e-4


def test_adjoint_is_transpose(orc):
    """orc.adjoint = -(1000/c^2) * L^T g, and <L s, g> = <s, L^T g>."""
    w = P.cfg_small(n_tx=24)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds)
    rp, col, val = orc.path_matrix(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"])
    gt = P.SplitMix64(7).normal(len(r["tof"]))
    LTg = np.zeros(w.grid.nx * w.grid.ny)
    rows = np.repeat(np.arange(len(gt)), np.diff(rp))
    np.add.at(LTg, col, val * gt[rows])
    gc = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"], gt).ravel()
    ref = -1000.0 * LTg / w.c.ravel() ** 2
    assert np.abs(gc - ref).max() <= 1e-12 * np.abs(ref).max()
    sv = P.SplitMix64(8).normal(LTg.size)
    Ls = np.add.reduceat(val * sv[col], rp[:-1])
    assert abs(Ls @ gt - sv @ LTg) <= 1e-12 * np.abs(Ls).sum() * np.abs(gt).max()


def test_adjoint_matches_central_differences(orc):
    """d(sum g_i T_i)/dc_j by central differences (h = 0.01 m/s) with the rays
    relinked tightly for every perturbed c, against the frozen-ray adjoint
    (Fermat): they agree to the discrete ray's stationarity residual. That
    residual is O(h^2) but not zero, because the ray equations use the
    interpolated grid gradient while T integrates the interpolated slowness;
    measured 4.2e-3 (L2 relative) here, against O(1) for a wrong sign, factor
    or index."""
    w = P.cfg_small(n_tx=32)
    base = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-10)
    gt = P.SplitMix64(9).normal(len(base["tof"]))
    gc = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, base["theta"], gt)
    x, y = w.grid.node_xy()
    inside = np.flatnonzero((x * x + y * y).ravel() < (0.8 * w.ring_radius) ** 2)
    rng = P.SplitMix64(10)
    picks = inside[(rng.uniform(8) * len(inside)).astype(int)]
    delta = 0.01
    fd = []
    for j in picks:
        J = []
        for sgn in (1, -1):
            c2 = w.c.copy().ravel()
            c2[j] += sgn * delta
            r2 = orc.link(w.grid, c2.reshape(w.c.shape), w.tx, w.ring_radius, w.ds, tol=1e-10,
                          theta0=base["theta"])
            J.append(r2["tof"] @ gt)
        fd.append((J[0] - J[1]) / (2 * delta))
    fd = np.array(fd)
    ad = gc.ravel()[picks]
    assert np.linalg.norm(fd - ad) <= 1e-2 * np.linalg.norm(ad), (fd, ad)


# ---------------------------------------------------------------- linking

def test_linked_root_inside_brute_force_bracket(orc):
    """Tiny case: a dense scan of the inward fan finds where the interception
    crosses the receiver; the linked angle must lie in that bracket."""
    g = P.Grid(32, 32, 0.5)
    R = 6.0
    tx = P.ring(8, R)
    c = P.gaussian_inclusions(g, seed=21, n_incl=2, amp=0.05, sigma_lo=1.0, sigma_hi=2.0,
                              centre_radius=3.0)
    pairs = P.all_pairs(8)
    ds = 0.1
    r = orc.link(g, c, tx, R, ds, tol=1e-7)
    assert (r["status"] == 0).all()
    n_scan = 801
    for k, (e, q) in enumerate(pairs):
        phi_e = np.arctan2(tx[e, 1], tx[e, 0])
        psi_r = np.mod(np.arctan2(tx[q, 1], tx[q, 0]) - phi_e, 2 * np.pi)
        th = phi_e + np.pi / 2 + np.linspace(0.01, np.pi - 0.01, n_scan)
        _, hit = orc.tof(g, c, tx, R, ds, th, pairs=np.repeat(pairs[k:k + 1], n_scan, 0))
        psi = np.mod(np.arctan2(hit[:, 1], hit[:, 0]) - phi_e, 2 * np.pi)
        m = psi - psi_r
        idx = np.flatnonzero(np.sign(m[:-1]) != np.sign(m[1:]))
        assert len(idx) == 1
        lo, hi = th[idx[0]], th[idx[0] + 1]
        t_link = phi_e + np.pi / 2 + np.mod(r["theta"][k] - phi_e - np.pi / 2, 2 * np.pi)
        assert lo <= t_link <= hi, (k, lo, t_link, hi)


def test_hits_land_on_ring_and_within_tol(orc):
    """Every linked interception lies on |x| = R (landing, Sec. 4.2's last point)
    and within tol of its receiver."""
    w = P.cfg_small(n_tx=32)
    pairs = P.all_pairs(32)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4)
    assert (r["status"] == 0).all()
    np.testing.assert_allclose(np.linalg.norm(r["hit"], axis=1), w.ring_radius, rtol=1e-12)
    assert np.linalg.norm(r["hit"] - w.tx[pairs[:, 1]], axis=1).max() <= 1e-4


def test_warm_start_reuses_angles(orc):
    """Sec. 3.4.1: later linearisations start from the previous angles; started
    from its own converged angles the oracle needs one trace per pair."""
    w = P.cfg_small(n_tx=24)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4)
    r2 = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, theta0=r["theta"])
    assert (r2["iters"] == 1).all()
    np.testing.assert_allclose(r2["tof"], r["tof"], rtol=1e-13)


def test_invalid_inputs_rejected(orc):
    g, tx, R = _small_ring(8)
    c = P.homogeneous(g)
    bad = c.copy()
    bad[3, 3] = -1.0
    with pytest.raises(ValueError):
        orc.link(g, bad, tx, R, 0.05)
    with pytest.raises(ValueError):
        orc.link(g, c, tx, 40.0, 0.05)          # ring outside the grid
    with pytest.raises(ValueError):
        orc.link(g, c, tx * 0.9, R, 0.05)       # transducers off the ring


# ---------------------------------------------------------------- fan start

def test_fan_start_reaches_the_same_rays(orc):
    """The fan-predicted cold start (an option) links the same rays as the
    straight-line start where the root is unique (weak inclusions), with fewer
    traces; the homogeneous medium links in one trace from the fan."""
    w = P.cfg_small(n_tx=32)
    a = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-9, fan_rays=0)
    b = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-9, fan_rays=64)
    assert (a["status"] == 0).all() and (b["status"] == 0).all()
    np.testing.assert_allclose(b["tof"], a["tof"], rtol=1e-11)
    assert np.abs(np.angle(np.exp(1j * (b["theta"] - a["theta"])))).max() < 1e-9
    assert b["iters"].mean() < a["iters"].mean()
    g, tx, R = _small_ring(32)
    h = orc.link(g, P.homogeneous(g), tx, R, 0.05, fan_rays=64)
    assert (h["iters"] == 1).all()


def test_fan_start_brute_force_bracket(orc):
    """With the fan start the linked angle still lies in the brute-force bracket."""
    g = P.Grid(32, 32, 0.5)
    R = 6.0
    tx = P.ring(8, R)
    c = P.gaussian_inclusions(g, seed=21, n_incl=2, amp=0.05, sigma_lo=1.0, sigma_hi=2.0, centre_radius=3.0)
    pairs = P.all_pairs(8)
    ds = 0.1
    r = orc.link(g, c, tx, R, ds, tol=1e-7, fan_rays=16)
    r0 = orc.link(g, c, tx, R, ds, tol=1e-7, fan_rays=0)
    assert (r["status"] == 0).all()
    d = np.angle(np.exp(1j * (r["theta"] - r0["theta"])))
    assert np.abs(d).max() < 1e-6


def test_fan_start_prediction_accuracy(orc):
    """The fan start's predictions are high order: on the 128^2 / 64-ring
    medium with 128 fan rays the first angle (inverse polynomial through the
    eight rays around the interval) links >= 90 % of the pairs to 1e-4 mm in
    one trace (measured 93.7 %; the four-ray cubic alone: 76.7 %); with 64 fan
    rays the second angle (inverse quartic through the first trace and four
    rays) leaves <= 1 % of the pairs needing a third trace (measured 0.1 %; the
    secant with the interval end: 8.0 %). The rays linked are the
    straight-start ones."""
    w = P.cfg_small()
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=128)
    assert (r["status"] == 0).all()
    assert (r["iters"] == 1).mean() >= 0.90, np.bincount(r["iters"])
    r64 = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=64)
    assert (r64["status"] == 0).all()
    assert (r64["iters"] >= 3).mean() <= 0.01, np.bincount(r64["iters"])
    r0 = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=0)
    np.testing.assert_allclose(r["tof"], r0["tof"], rtol=1e-8)


def test_fan_step_changes_only_the_predictions(orc):
    """The fan may be traced at its own step (fan_ds): fan_ds = ds is the
    default exactly; a coarse fan (h/2 = 5 ds) links the same rays as the
    straight-line start and keeps the predictions high order (>= 85 % of the
    pairs in one trace with 128 rays); in a homogeneous medium (straight rays,
    exact for any step) every pair still links in one trace from a fan traced
    at 10 ds, which holds only while the fan's launch angles follow ds, the
    step the predictions assume."""
    w = P.cfg_small()
    a = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=128)
    b = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=128, fan_ds=w.ds)
    for k in ("theta", "tof", "iters"):
        np.testing.assert_array_equal(a[k], b[k])
    c = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=128, fan_ds=0.5 * w.grid.h)
    assert (c["status"] == 0).all()
    r0 = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=0)
    np.testing.assert_allclose(c["tof"], r0["tof"], rtol=1e-8)
    assert (c["iters"] == 1).mean() >= 0.85, np.bincount(c["iters"])
    assert not np.array_equal(c["theta"], a["theta"])   # the coarse fan is traced: other first angles
    g, tx, R = _small_ring(32)
    h = orc.link(g, P.homogeneous(g), tx, R, 0.05, fan_rays=64, fan_ds=0.5)
    assert (h["iters"] == 1).all()
    with pytest.raises(Exception):
        orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, fan_rays=64, fan_ds=-1.0)


def test_subfan_refines_only_the_third_angle(orc):
    """R12: after a second missed trace, a sub-fan inside the bracket predicts
    the third angle. subfan = 0 is the plain rule exactly. On the 128^2 /
    64-ring case with a coarse 16-ray fan (many pairs reach a third trace) the
    sub-fan links the same rays as the straight-line start (ToF within 1e-8),
    changes nothing before the third trace, and with 16 rays links at least
    90 % of the pairs that make a third trace at that trace (79 % without it,
    where the third angle is a secant step), halving the pairs that need four
    or more."""
    w = P.cfg_small()
    kw = dict(tol=1e-4, fan_rays=16, fan_ds=0.5 * w.grid.h)
    r0 = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=1e-4, fan_rays=0)
    a = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, subfan=0, **kw)
    b = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, **kw)
    for k in ("theta", "tof", "iters"):
        np.testing.assert_array_equal(a[k], b[k])
    s = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, subfan=16, **kw)
    assert (s["status"] == 0).all()
    np.testing.assert_allclose(s["tof"], r0["tof"], rtol=1e-8)
    early = a["iters"] <= 2
    np.testing.assert_array_equal(s["theta"][early], a["theta"][early])
    np.testing.assert_array_equal(s["iters"][early], a["iters"][early])
    third = s["iters"] >= 3
    assert third.sum() > 1000
    at3 = float(np.mean(s["iters"][third] == 3))
    assert at3 >= 0.90, (at3, np.bincount(s["iters"]))
    assert (s["iters"] >= 4).sum() <= 0.5 * (a["iters"] >= 4).sum(), (np.bincount(s["iters"]), np.bincount(a["iters"]))
    with pytest.raises(Exception):
        orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, subfan=-1, **kw)


def test_subfan_angles_evenly_inside(orc):
    """R12's sub-fan: M rays evenly spaced strictly inside the bracket, in the
    direction from the end of negative misfit (either orientation)."""
    for ta, tb, M in ((0.2, 1.0, 8), (3.0, 2.5, 4), (-1.0, 1.0, 1)):
        th = orc.subfan_angles(ta, tb, M)
        step = (tb - ta) / (M + 1)
        np.testing.assert_allclose(np.diff(np.r_[ta, th, tb]), step, rtol=0, atol=1e-14)


def _cubic_inverse(coef, theta):
    """m with theta(m) = coef[0] + coef[1] m + coef[2] m^2 + coef[3] m^3 (the
    real root; theta(m) monotone)."""
    out = []
    for t in np.atleast_1d(theta):
        r = np.roots([coef[3], coef[2], coef[1], coef[0] - t])
        out.append(r[np.argmin(np.abs(r.imag))].real)
    return np.array(out)


def test_subfan_prediction_exact_for_cubic_inverse(orc):
    """The third angle is the root of the inverse cubic through the four
    sub-fan rays around the interval: exact (to rounding) when the angle is a
    cubic polynomial of the misfit, in both orientations. The bracket ends,
    whose misfits may carry the Illinois halving, never enter it: here they
    are set off the curve, and a root next to an end gives the Regula-Falsi
    point of its interval instead."""
    for coef, ta_m, tb_m in (((0.3, 0.8, 0.2, 0.05), -1.6, 1.2), ((0.3, -0.8, 0.2, -0.05), -1.0, 1.6)):
        ta, tb = np.polyval(coef[::-1], ta_m), np.polyval(coef[::-1], tb_m)
        for M in (4, 8):
            th = orc.subfan_angles(ta, tb, M)
            m = _cubic_inverse(coef, th)
            seq_t = np.r_[ta, th, tb]
            seq_m = np.r_[0.5 * ta_m, m, 0.5 * tb_m]        # ends off the curve
            j = int(np.argmax(seq_m >= 0))
            assert 3 <= j <= M - 1                            # four sub-fan rays around the root
            c3 = 0.5 * (seq_t[j - 1] + seq_t[j])                   # the plain rule's candidate
            p = orc.subfan_predict(seq_t, seq_m, np.arange(M + 2), c3, R=10.0)
            assert p["refined"]
            assert p["changes_sign"]
            assert (p["ta"], p["tb"]) == (seq_t[j - 1], seq_t[j])
            assert abs(p["theta3"] - coef[0]) <= 1e-12, (M, p["theta3"])
    # the root between the first two sub-fan rays: the four around it would take
    # the bracket end (off the curve), so the Regula-Falsi point
    coef = (0.3, 0.8, 0.2, 0.05)
    ta_m, tb_m = -1.0, 1.5
    ta, tb = np.polyval(coef[::-1], ta_m), np.polyval(coef[::-1], tb_m)
    th = orc.subfan_angles(ta, tb, 4)
    m = _cubic_inverse(coef, th)
    seq_t, seq_m = np.r_[ta, th, tb], np.r_[0.5 * ta_m, m, 0.5 * tb_m]
    j = int(np.argmax(seq_m >= 0))
    assert j == 2, seq_m
    p = orc.subfan_predict(seq_t, seq_m, [0, 1, 2, 3, 4, 5], seq_t[1], R=10.0)
    rf = seq_t[1] - seq_m[1] * (seq_t[2] - seq_t[1]) / (seq_m[2] - seq_m[1])
    assert (p["ta"], p["tb"]) == (seq_t[1], seq_t[2]) and abs(p["theta3"] - rf) <= 1e-15
    # the root between the last sub-fan ray and the far end: linear
    ta_m, tb_m = -2.0, 0.05
    ta, tb = np.polyval(coef[::-1], ta_m), np.polyval(coef[::-1], tb_m)
    th = orc.subfan_angles(ta, tb, 4)
    m = _cubic_inverse(coef, th)
    assert (m < 0).all()
    seq_t, seq_m = np.r_[ta, th, tb], np.r_[0.5 * ta_m, m, 0.5 * tb_m]
    p = orc.subfan_predict(seq_t, seq_m, [0, 1, 2, 3, 4, 5], tb, R=10.0)
    rf = seq_t[4] - seq_m[4] * (seq_t[5] - seq_t[4]) / (seq_m[5] - seq_m[4])
    assert (p["ta"], p["tb"]) == (seq_t[4], seq_t[5]) and abs(p["theta3"] - rf) <= 1e-15


def test_subfan_picks_the_crossing_at_the_plain_candidate(orc):
    """Several sign changes in the sequence, one of them a jump of about 2 pi R
    (the hit wrapping around the emitter): the bracket is the crossing (sign
    change by less than pi R between entries with no missing ray between them)
    that holds the plain rule's third angle c3, with
    either orientation; without four sub-fan rays around it the third angle is
    its Regula-Falsi point; the secant starts from its end of smaller |misfit|;
    when no crossing holds c3, nothing is refined and c3 is traced."""
    t = np.array([0.0, 0.1, 0.2, 0.3, 0.4, 0.5])
    m = np.array([-1.0, -0.5, 0.3, -0.2, 0.6, 1.0])
    p = orc.subfan_predict(t, m, [0, 1, 2, 3, 4, 5], 0.13, R=1.0)
    assert p["refined"] and (p["ta"], p["tb"]) == (0.1, 0.2) and p["changes_sign"]
    assert abs(p["theta3"] - (0.1 + 0.5 * 0.1 / 0.8)) <= 1e-15
    assert (p["start_theta"], p["start_m"]) == (0.2, 0.3)
    q = orc.subfan_predict(t, m, [0, 1, 2, 3, 4, 5], 0.27, R=1.0)          # the falling crossing (0.2, 0.3)
    assert q["refined"] and (q["ta"], q["tb"]) == (0.3, 0.2) and q["changes_sign"]
    assert abs(q["theta3"] - (0.3 - (-0.2) * (0.2 - 0.3) / (0.3 + 0.2))) <= 1e-15
    assert (q["start_theta"], q["start_m"]) == (0.3, -0.2)
    r = orc.subfan_predict(t, m, [0, 1, 2, 3, 4, 5], 0.46, R=1.0)          # no crossing in (0.4, 0.5)
    assert not r["refined"] and r["theta3"] == 0.46 and (r["ta"], r["tb"]) == (0.0, 0.5)
    mj = np.array([-1.0, -1.5, 2.0, -0.1, 0.2, 1.0])                        # jump of 3.5 > pi at (0.1, 0.2)
    j = orc.subfan_predict(t, mj, [0, 1, 2, 3, 4, 5], 0.15, R=1.0)
    assert not j["refined"] and j["theta3"] == 0.15
    j2 = orc.subfan_predict(t, mj, [0, 1, 2, 3, 4, 5], 0.15, R=2.0)        # the same sign change, 3.5 < 2 pi
    assert j2["refined"] and (j2["ta"], j2["tb"]) == (0.1, 0.2)
    k = orc.subfan_predict(t, mj, [0, 1, 2, 3, 4, 5], 0.34, R=1.0)
    assert k["refined"] and (k["ta"], k["tb"]) == (0.3, 0.4)
    # a ray that missed the ring between two entries: their sign change is no crossing
    g = orc.subfan_predict([0.0, 0.1, 0.3, 0.4, 0.5], [-1.0, -0.5, 0.3, 0.6, 1.0], [0, 1, 3, 4, 5], 0.2, R=1.0)
    assert not g["refined"] and g["theta3"] == 0.2
    g2 = orc.subfan_predict([0.0, 0.1, 0.2, 0.4, 0.5], [-1.0, -0.5, 0.3, 0.6, 1.0], [0, 1, 2, 4, 5], 0.15, R=1.0)
    assert g2["refined"] and (g2["ta"], g2["tb"]) == (0.1, 0.2)
    # strictly falling misfits around the root: the inverse cubic applies too
    coef = (0.3, -0.8, 0.2, -0.05)
    th = np.array([0.0, 0.15, 0.25, 0.35, 0.45, 0.6])
    mm = _cubic_inverse(coef, th)
    assert (np.diff(mm) < 0).all()
    assert int(np.argmax(mm < 0)) == 3
    c = orc.subfan_predict(th, mm, [0, 1, 2, 3, 4, 5], 0.31, R=10.0)
    assert c["refined"] and abs(c["theta3"] - coef[0]) <= 1e-12, c
