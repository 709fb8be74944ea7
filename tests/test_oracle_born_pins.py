"""Pins of the FP64 ray-Born oracle (fan maps with paraxial rays, Born map and
its adjoint) against closed forms and invariants, none of which reuses the
oracle's own formulas: straight rays and circular arcs solve the ray and
paraxial equations exactly, finite differences of neighbouring fan rays give
the ray Jacobian independently of the paraxial system (the paper's auxiliary
rays, Sec. 3.5), Fermat's principle ties the maps to the separately pinned
two-point linking, and a point scatterer in a homogeneous medium has a closed
Born response. The mutation tests show that plausible slips fail one of them.
"""
import numpy as np
import pytest

from paper_2511_18511_gb300 import phantoms as P

C0 = 1.5  # mm/us


def _homog(n=64, h=0.5, R=14.0, n_tx=8):
    g = P.Grid(n, n, h)
    return g, P.homogeneous(g), P.ring(n_tx, R), R


# ------------------------------------------------------------ single fan rays

def test_fan_ray_homogeneous_straight(orc):
    """c = const: the ray is straight, Q is the distance travelled, P = 1/c,
    T = distance / c."""
    g, c, tx, R = _homog()
    r = orc.fan_ray(g, c, R, tx[0], np.pi + 0.3, 0.05)
    dist = np.hypot(r["x"] - tx[0, 0], r["y"] - tx[0, 1])
    assert len(dist) > 100
    np.testing.assert_allclose(r["Q"], dist, atol=1e-11)
    np.testing.assert_allclose(r["P"], 1.0 / C0, rtol=1e-14)
    np.testing.assert_allclose(r["T"], dist / C0, atol=1e-12)
    np.testing.assert_allclose(r["dx"], np.cos(np.pi + 0.3), atol=1e-14)


@pytest.mark.parametrize("theta_off", [0.2, -0.5, 0.8])
def test_fan_ray_linear_gradient_closed_form_Q(orc, theta_off):
    """c = c_m + g y: the Hessian vanishes, so P = 1/c_t stays constant and
    Q = int c ds / c_t. Along the circular ray, c ds = g rho^2 sin(phi) dphi
    integrates to g rho |dx|, and rho = c_t / (g |cos a|) (Snell), so
    Q = |x - x_e| / |cos a| with a the launch angle to the x axis."""
    g = P.Grid(128, 128, 0.5)
    c = P.linear_gradient(g)
    tx = P.ring(16, 30.0)
    th = np.pi + theta_off
    r = orc.fan_ray(g, c, 30.0, tx[0], th, 0.05)
    q = np.abs(r["x"] - tx[0, 0]) / abs(np.cos(th))
    np.testing.assert_allclose(r["Q"][1:], q[1:], rtol=1e-10)
    c_t = 1e-3 * (1500.0 + tx[0, 1])
    np.testing.assert_allclose(r["P"], 1.0 / c_t, rtol=1e-12)


@pytest.mark.parametrize("k,off", [(0, 0.1), (9, -0.6), (18, 0.9), (40, -0.25)])
def test_paraxial_Q_matches_auxiliary_rays(orc, k, off):
    """The paper's auxiliary-ray Jacobian (Sec. 3.5): two rays launched at
    theta +- delta; their separation along the normal n of the reference ray,
    divided by 2 delta, is dq/dtheta, which the paraxial Q (Q(0) = 0,
    P(0) = 1/c_t) equals to first order. Broad Gaussian inclusions; the
    remaining gap is the bilinear Hessian against the derivative of the
    bilinear gradient, O(h^2)."""
    w = P.cfg_born_small()
    e = w.tx[k]
    th = np.arctan2(e[1], e[0]) + np.pi + off
    d = 1e-6
    a = orc.fan_ray(w.grid, w.c, w.ring_radius, e, th, w.ds)
    p = orc.fan_ray(w.grid, w.c, w.ring_radius, e, th + d, w.ds)
    m = orc.fan_ray(w.grid, w.c, w.ring_radius, e, th - d, w.ds)
    n = min(len(a["x"]), len(p["x"]), len(m["x"]))
    q = (-a["dy"][:n] * (p["x"][:n] - m["x"][:n]) + a["dx"][:n] * (p["y"][:n] - m["y"][:n])) / (2 * d)
    assert n > 200
    err = np.abs(a["Q"][1:n] - q[1:n]).max() / np.abs(q[1:n]).max()
    assert err < 2e-3, err


# ------------------------------------------------------------------- the maps

def test_maps_homogeneous_match_distance(orc):
    """Homogeneous medium: every node inside the ring is reached, T = r/c up to
    the remainder of the second-order extrapolation from the foot of the
    node on the nearest ray (|T - r/c| <= 0.01 s h^3 / r^2 for r >= 2h; an
    extrapolation from the sample instead of the foot leaves ~0.05) and
    A = 1/sqrt(r) of the nearest ray (|A sqrt(r) - 1| <= 0.005 h / r)."""
    g, c, tx, R = _homog()
    K = P.born_fan_rays(R, g.h)
    T, A = orc.fan_maps(g, c, tx, R, 0.05, K)
    x, y = g.node_xy()
    inside = x * x + y * y < R * R
    for t in range(len(tx)):
        r = np.hypot(x - tx[t, 0], y - tx[t, 1])
        assert np.isfinite(T[t][inside]).all() and (A[t][inside] > 0).all()
        m = inside & (r >= 2 * g.h)
        assert (np.abs(T[t][m] - r[m] / C0) <= 0.01 * g.h ** 3 / (C0 * r[m] ** 2)).all()
        assert (np.abs(A[t][m] * np.sqrt(r[m]) - 1.0) <= 0.005 * g.h / r[m]).all()
        assert np.isinf(T[t][x * x + y * y > (R + 2 * g.h) ** 2]).all()


def test_maps_fermat_against_linking(orc):
    """Fermat: for first-arrival maps, min_x T_e(x) + T_r(x) is the two-point
    travel time, which the separately pinned linking oracle computes. Pairs at
    least 8 elements apart (the node lattice misses the ray by < h, a
    second-order excess that is relatively small on long rays)."""
    w = P.cfg_born_small()
    T, _ = orc.fan_maps(w.grid, w.c, w.tx, w.ring_radius, w.ds, w.fan_rays)
    x, y = w.grid.node_xy()
    inside = x * x + y * y < w.ring_radius ** 2
    assert np.isfinite(T[:, inside]).all()
    pairs = P.all_pairs(w.n_tx)
    sep = np.abs(pairs[:, 0] - pairs[:, 1])
    sep = np.minimum(sep, w.n_tx - sep)
    sel = np.flatnonzero(sep >= 8)[::23]
    L = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, pairs=pairs[sel], fan_rays=256)
    rel = np.array([(T[e] + T[r])[inside].min() / L["tof"][k] - 1 for k, (e, r) in enumerate(pairs[sel])])
    assert rel.min() >= -2e-4 and rel.max() <= 5e-4, (rel.min(), rel.max())


def test_maps_match_brute_force_over_all_fan_samples(orc):
    """Tiny heterogeneous case: every map entry of a few nodes recomputed by
    brute force from the recorded samples of every fan ray (the per-sample
    candidates of the map rule, the earliest for T, the least
    T + eta (b/h)^2 for A), independently of the map routine's loops."""
    g = P.Grid(48, 48, 0.5)
    R = 10.0
    c = P.gaussian_inclusions(g, 31, amp=0.05, sigma_lo=2.0, sigma_hi=3.0, centre_radius=5.0)
    tx = P.ring(3, R)
    ds, K, eta = 0.05, P.born_fan_rays(R, g.h), orc.ETA
    T, A = orc.fan_maps(g, c, tx, R, ds, K)
    x, y = g.node_xy()
    rng = P.SplitMix64(32)
    inside = np.flatnonzero((x * x + y * y).ravel() < (R - 1.0) ** 2)
    nodes = inside[(rng.uniform(12) * len(inside)).astype(int)]
    h = g.h
    for t in range(len(tx)):
        a_min, step = orc.fan_angles(tx[t], R, ds, K)
        c_t = orc.sample(g, c, tx[t][None, :])[0, 0]
        best = {int(k): (np.inf, np.inf, 0.0) for k in nodes}      # T, score, A
        for k in range(K):
            r = orc.fan_ray(g, c, R, tx[t], a_min + k * step, ds)
            sl = slice(1, None)                                      # the transducer itself offers nothing
            X, Y, DX, DY = r["x"][sl], r["y"][sl], r["dx"][sl], r["dy"][sl]
            ic = np.floor((X - g.x0) / h + 0.5).astype(int)
            jc = np.floor((Y - g.y0) / h + 0.5).astype(int)
            for node in nodes:
                j, i = divmod(int(node), g.nx)
                m = np.flatnonzero((np.abs(ic - i) <= 1) & (np.abs(jc - j) <= 1))
                if len(m) == 0:
                    continue
                Dx, Dy = g.x0 + i * h - X[m], g.y0 + j * h - Y[m]
                al = DX[m] * Dx + DY[m] * Dy
                ac = -DY[m] * Dx + DX[m] * Dy
                ok = (al >= -0.5 * ds) & (al < 0.5 * ds)
                if not ok.any():
                    continue
                m, al, ac = m[ok], al[ok], ac[ok]
                Q, Pp, cc, ss, Tm = (r[f][sl][m] for f in ("Q", "P", "c", "s", "T"))
                Qf = Q + al * cc * Pp
                Qc = np.where(np.abs(Qf) >= h, Qf, np.where(Qf < 0, -h, h))
                curv = Pp / Qf
                curv = np.where(curv >= 0, curv, Pp / Qc)
                cand = Tm + ss * al + 0.5 * curv * ac * ac
                amp = np.sqrt(cc / (c_t * np.abs(Qc)))
                score = cand + eta * (ac / h) ** 2
                T0, S0, A0 = best[int(node)]
                q = int(np.argmin(score))
                best[int(node)] = (min(T0, cand.min()), min(S0, score[q]),
                                   amp[q] if score[q] < S0 else A0)
        for node in nodes:
            j, i = divmod(int(node), g.nx)
            Tb, _, Ab = best[int(node)]
            assert abs(T[t, j, i] - Tb) <= 1e-12 * Tb, (t, node, T[t, j, i], Tb)
            assert abs(A[t, j, i] - Ab) <= 1e-12 * Ab, (t, node, A[t, j, i], Ab)


# --------------------------------------------------------- Born map and adjoint

def _synthetic_maps(g, tx, seed):
    """Seeded smooth maps: straight-ray times plus a random ripple, 1/sqrt(r)."""
    x, y = g.node_xy()
    rng = P.SplitMix64(seed)
    T = np.empty((len(tx), g.ny, g.nx))
    A = np.empty_like(T)
    for t in range(len(tx)):
        r = np.hypot(x - tx[t, 0], y - tx[t, 1]) + 0.1
        T[t] = r / C0 + 0.05 * rng.normal(x.size).reshape(x.shape)
        A[t] = 1.0 / np.sqrt(r)
    T[1, 3, 4] = np.inf            # an unreached node
    A[1, 3, 4] = 0.0
    return T, A


def test_born_dot_product_identity(orc):
    """Re<F dc, d> = <dc, F* d> for seeded random dc and complex d."""
    g = P.Grid(24, 24, 0.5)
    R = 5.5
    tx = P.ring(6, R)
    T, A = _synthetic_maps(g, tx, 3)
    f = P.born_frequencies(3)
    rng = P.SplitMix64(4)
    dc = rng.normal(g.nx * g.ny).reshape(g.ny, g.nx)
    d = (rng.normal(3 * 36) + 1j * rng.normal(3 * 36)).reshape(3, 6, 6)
    lhs = np.sum(np.real(np.conj(orc.born_apply(g, R, T, A, f, dc)) * d))
    rhs = np.sum(dc * orc.born_adjoint(g, R, T, A, f, d))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(dc)) * np.abs(d).sum() * 100, (lhs, rhs)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_born_point_scatterer_homogeneous(orc):
    """One node x0 perturbed by dc in a homogeneous medium: the Born data are
    omega^2 h^2 dc exp(i omega (r_e + r_r)/c) / sqrt(r_e r_r) (2D ray Green's
    functions A = 1/sqrt(r), phase omega r / c), zero on the diagonal."""
    g, c, tx, R = _homog()
    T, A = orc.fan_maps(g, c, tx, R, 0.05, P.born_fan_rays(R, g.h))
    x, y = g.node_xy()
    j0, i0 = 30, 37
    dc = np.zeros_like(c)
    dc[j0, i0] = 3.0
    f = P.born_frequencies(4)
    d = orc.born_apply(g, R, T, A, f, dc)
    rx = np.hypot(x[j0, i0] - tx[:, 0], y[j0, i0] - tx[:, 1])
    for k, fm in enumerate(f):
        om = 2 * np.pi * fm
        want = om ** 2 * g.h ** 2 * 3.0 * np.exp(1j * om * (rx[:, None] + rx[None, :]) / C0) / np.sqrt(
            rx[:, None] * rx[None, :])
        np.fill_diagonal(want, 0.0)
        assert np.all(np.diag(d[k]) == 0)
        err = np.abs(d[k] - want)
        bound = np.abs(want) * (0.1 * g.h / np.minimum(rx[:, None], rx[None, :]) + 1e-6)
        assert (err <= bound).all(), (err / np.maximum(np.abs(want), 1e-300)).max()


def test_born_adjoint_single_datum_homogeneous(orc):
    """Adjoint of one datum d[f][e][r] = 1 in a homogeneous medium:
    omega^2 h^2 cos(omega (r_e + r_r)/c) / sqrt(r_e r_r) at every node inside
    the ring, 0 outside."""
    g, c, tx, R = _homog()
    T, A = orc.fan_maps(g, c, tx, R, 0.05, P.born_fan_rays(R, g.h))
    f = P.born_frequencies(2)
    d = np.zeros((2, len(tx), len(tx)), complex)
    d[1, 2, 5] = 1.0
    out = orc.born_adjoint(g, R, T, A, f, d)
    x, y = g.node_xy()
    inside = x * x + y * y < R * R
    re = np.hypot(x - tx[2, 0], y - tx[2, 1])
    rr = np.hypot(x - tx[5, 0], y - tx[5, 1])
    om = 2 * np.pi * f[1]
    want = om ** 2 * g.h ** 2 * np.cos(om * (re + rr) / C0) / np.sqrt(re * rr)
    m = inside & (re >= 2 * g.h) & (rr >= 2 * g.h)
    amp = om ** 2 * g.h ** 2 / np.sqrt(re * rr)
    assert (np.abs(out[m] - want[m]) <= amp[m] * (0.1 * g.h / np.minimum(re, rr)[m] + 1e-6)).all()
    assert (out[~inside] == 0).all()


def linear_gradient_maps_closed_form(g, grad, tx):
    """Closed forms of the maps in c = 1500 + grad y (m/s, y in mm): the ray
    from x_e to a node is the circle through both centred on y = -1500/grad;
    T = arccosh(1 + grad^2 r^2 / (2 c_e c)) / grad and, with the Hessian zero,
    Q = int c ds / c_e = |x - x_e| / |cos a| (a the launch angle to the x axis,
    cos a = (y_e + 1500/grad) / rho), A = sqrt(c / (c_e max(Q, h)))."""
    x, y = g.node_xy()
    xe, ye = tx
    r = np.hypot(x - xe, y - ye)
    gk = 1e-3 * grad                                    # (mm/us) per mm
    ce, cn = 1e-3 * (1500.0 + grad * ye), 1e-3 * (1500.0 + grad * y)
    T = np.arccosh(1.0 + gk * gk * r * r / (2.0 * ce * cn)) / gk
    y0 = 1500.0 / grad
    with np.errstate(divide="ignore", invalid="ignore"):
        xc = ((x * x - xe * xe) + ((y + y0) ** 2 - (ye + y0) ** 2)) / (2.0 * (x - xe))
    rho = np.hypot(xe - xc, ye + y0)
    Q = np.abs(x - xe) * rho / np.abs(ye + y0)
    A = np.sqrt(cn / (ce * np.maximum(Q, g.h)))
    return T, A, r, np.abs(x - xe)


@pytest.mark.parametrize("grad,tol_t,tol_a", [(1.0, 2e-6, 5e-5), (5.0, 2e-5, 1.5e-4)])
def test_maps_linear_gradient_closed_form(orc, grad, tol_t, tol_a):
    """Refracting medium c = 1500 + grad y (no caustics): the maps' travel times
    and amplitudes against the closed forms of the circular rays (B3-B5 in a
    medium where c(x) differs from c_t and rays bend): T within tol_t and A
    within tol_a relative at every inside node at least 2h from the transducer
    (and from its vertical, where |x - x_e| / |cos a| loses precision); the
    error grows with the ray curvature, which the extrapolation from the foot
    of the node neglects."""
    g = P.Grid(64, 64, 0.5)
    R = 14.0
    c = P.linear_gradient(g, 1500.0, grad)
    tx = P.ring(8, R)
    T, A = orc.fan_maps(g, c, tx, R, 0.05, P.born_fan_rays(R, g.h))
    x, y = g.node_xy()
    inside = x * x + y * y < R * R
    for t in range(len(tx)):
        Tc, Ac, r, adx = linear_gradient_maps_closed_form(g, grad, tx[t])
        m = inside & (r >= 2 * g.h) & (adx > 2 * g.h)
        eT = np.abs(T[t][m] / Tc[m] - 1)
        eA = np.abs(A[t][m] / Ac[m] - 1)
        assert eT.max() <= tol_t and eA.max() <= tol_a, (t, eT.max(), eA.max())
