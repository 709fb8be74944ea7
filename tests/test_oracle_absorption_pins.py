"""Pins of the oracle's absorption in the ray-Born Green's functions (paper
Appendix: complex wavenumber k + i alpha with alpha = alpha0 omega^y, the
absorption amplitude accumulated along the ray, A = A_geom A_abs).

Independent checks: the path integral of a uniform alpha0 along the straight
rays of a homogeneous medium (alpha0 times the distance to the foot of the
node on its ray); a brute-force recomputation, in numpy from the recorded fan
samples, of the path integral of a linear alpha0 field (which bilinear
sampling reproduces exactly) for a few nodes of a heterogeneous medium; the
closed-form Born response of a point scatterer in a homogeneous absorbing
medium at several frequencies (the power law's frequency dependence); the
dot-product identity with absorption; and alpha0 = 0 reproducing the maps and
data without absorption exactly.
"""
import numpy as np

from paper_2511_18511_gb300 import phantoms as P

from .test_oracle_born_pins import C0, _homog, _synthetic_maps

Y = 1.3          # power-law exponent (soft tissue: 1 < y <= 1.5)
ALPHA0 = 2.0e-8  # Np (rad/s)^-y m^-1: ~1 Np over 10 cm at 1 MHz for y = 1.3


def _omega_s_pow(f_mhz, y=Y):
    return (2 * np.pi * np.asarray(f_mhz) * 1e6) ** y


def test_absorption_uniform_alpha_homogeneous(orc):
    """Uniform alpha0 in a homogeneous medium: Lam = alpha0 (r - b^2/(2r)) with
    b the node's distance to the straight ray that supplies A (<= h/2), in
    metres; unreached nodes 0."""
    g, c, tx, R = _homog()
    K = P.born_fan_rays(R, g.h)
    al = np.full_like(c, ALPHA0)
    T, A, L = orc.fan_maps(g, c, tx, R, 0.05, K, alpha0=al)
    T0, A0 = orc.fan_maps(g, c, tx, R, 0.05, K)
    np.testing.assert_array_equal(T, T0)
    np.testing.assert_array_equal(A, A0)
    x, y = g.node_xy()
    inside = x * x + y * y < R * R
    for t in range(len(tx)):
        r = np.hypot(x - tx[t, 0], y - tx[t, 1])
        m = inside & (r >= 2 * g.h)
        dist = L[t][m] / (1e-3 * ALPHA0)
        assert (dist <= r[m] + 1e-9).all() and (dist >= r[m] - g.h ** 2 / (8 * r[m]) - 1e-9).all()
        assert (L[t][~np.isfinite(T[t])] == 0).all()


def test_absorption_linear_alpha_brute_force(orc):
    """Heterogeneous c, alpha0 = a + g x (reproduced exactly by bilinear
    sampling): for a few nodes, Lam is recomputed from the recorded samples of
    every fan ray (trapezoid of alpha0 over the samples, plus alpha0 a from the
    sample to the node's foot, for the candidate of least T + eta (b/h)^2)."""
    g = P.Grid(48, 48, 0.5)
    R = 10.0
    c = P.gaussian_inclusions(g, 31, amp=0.05, sigma_lo=2.0, sigma_hi=3.0, centre_radius=5.0)
    x, y = g.node_xy()
    a0, gx = 3.0e-8, 1.5e-9
    al = a0 + gx * x
    assert (al > 0).all()
    tx = P.ring(3, R)
    ds, K, eta = 0.05, P.born_fan_rays(R, g.h), orc.ETA
    T, A, L = orc.fan_maps(g, c, tx, R, ds, K, alpha0=al)
    rng = P.SplitMix64(32)
    inside = np.flatnonzero((x * x + y * y).ravel() < (R - 1.0) ** 2)
    nodes = inside[(rng.uniform(12) * len(inside)).astype(int)]
    h = g.h
    for t in range(len(tx)):
        a_min, step = orc.fan_angles(tx[t], R, ds, K)
        c_t = orc.sample(g, c, tx[t][None, :])[0, 0]
        best = {int(k): (np.inf, 0.0) for k in nodes}      # score, Lam
        for k in range(K):
            r = orc.fan_ray(g, c, R, tx[t], a_min + k * step, ds)
            alpha = a0 + gx * r["x"]
            Lam = 1e-3 * np.concatenate([[0.0], np.cumsum(0.5 * ds * (alpha[1:] + alpha[:-1]))])
            sl = slice(1, None)
            X, Y_, DX, DY = r["x"][sl], r["y"][sl], r["dx"][sl], r["dy"][sl]
            ic = np.floor((X - g.x0) / h + 0.5).astype(int)
            jc = np.floor((Y_ - g.y0) / h + 0.5).astype(int)
            for node in nodes:
                j, i = divmod(int(node), g.nx)
                m = np.flatnonzero((np.abs(ic - i) <= 1) & (np.abs(jc - j) <= 1))
                if len(m) == 0:
                    continue
                Dx, Dy = g.x0 + i * h - X[m], g.y0 + j * h - Y_[m]
                along = DX[m] * Dx + DY[m] * Dy
                across = -DY[m] * Dx + DX[m] * Dy
                ok = (along >= -0.5 * ds) & (along < 0.5 * ds)
                if not ok.any():
                    continue
                m, along, across = m[ok], along[ok], across[ok]
                Q, Pp, cc, ss, Tm = (r[f][sl][m] for f in ("Q", "P", "c", "s", "T"))
                Qf = Q + along * cc * Pp
                Qc = np.where(np.abs(Qf) >= h, Qf, np.where(Qf < 0, -h, h))
                curv = Pp / Qf
                curv = np.where(curv >= 0, curv, Pp / Qc)
                score = Tm + ss * along + 0.5 * curv * across * across + eta * (across / h) ** 2
                amp = np.sqrt(cc / (c_t * np.abs(Qc)))
                q = int(np.lexsort((amp, score))[0])
                if score[q] < best[int(node)][0]:
                    best[int(node)] = (score[q], Lam[sl][m][q] + 1e-3 * alpha[sl][m][q] * along[q])
        for node in nodes:
            j, i = divmod(int(node), g.nx)
            Lb = best[int(node)][1]
            assert abs(L[t, j, i] - Lb) <= 1e-12 * Lb, (t, node, L[t, j, i], Lb)


def test_absorption_point_scatterer_homogeneous(orc):
    """One perturbed node in a homogeneous medium with uniform alpha0: the Born
    data are omega^2 h^2 dc exp(-omega_s^y alpha0 (r_e + r_r)) exp(i omega
    (r_e + r_r)/c) / sqrt(r_e r_r), so the decay follows the power law in f."""
    g, c, tx, R = _homog()
    al = np.full_like(c, ALPHA0)
    T, A, L = orc.fan_maps(g, c, tx, R, 0.05, P.born_fan_rays(R, g.h), alpha0=al)
    x, y = g.node_xy()
    j0, i0 = 30, 37
    dc = np.zeros_like(c)
    dc[j0, i0] = 3.0
    f = np.array([0.5, 1.0, 2.0, 4.0])
    d = orc.born_apply(g, R, T, A, f, dc, Lam=L, y=Y)
    rx = np.hypot(x[j0, i0] - tx[:, 0], y[j0, i0] - tx[:, 1])
    rs = rx[:, None] + rx[None, :]
    decay_seen = []
    for k, fm in enumerate(f):
        om = 2 * np.pi * fm
        att = np.exp(-_omega_s_pow(fm) * ALPHA0 * 1e-3 * rs)
        want = om ** 2 * g.h ** 2 * 3.0 * att * np.exp(1j * om * rs / C0) / np.sqrt(rx[:, None] * rx[None, :])
        np.fill_diagonal(want, 0.0)
        err = np.abs(d[k] - want)
        bound = np.abs(want) * (0.1 * g.h / np.minimum(rx[:, None], rx[None, :]) + 1e-6)
        assert (err <= bound).all(), (err / np.maximum(np.abs(want), 1e-300)).max()
        decay_seen.append(att.min())
    assert decay_seen[-1] < 0.1 and decay_seen[0] > 0.8    # the law matters over this band


def test_absorption_dot_product_identity(orc):
    """Re<F dc, d> = <dc, F* d> with absorption factors in E."""
    g = P.Grid(24, 24, 0.5)
    R = 5.5
    tx = P.ring(6, R)
    T, A = _synthetic_maps(g, tx, 3)
    rng = P.SplitMix64(9)
    L = 1e-8 * np.abs(rng.normal(T.size)).reshape(T.shape)
    f = P.born_frequencies(3)
    dc = rng.normal(g.nx * g.ny).reshape(g.ny, g.nx)
    d = (rng.normal(3 * 36) + 1j * rng.normal(3 * 36)).reshape(3, 6, 6)
    lhs = np.sum(np.real(np.conj(orc.born_apply(g, R, T, A, f, dc, Lam=L, y=Y)) * d))
    rhs = np.sum(dc * orc.born_adjoint(g, R, T, A, f, d, Lam=L, y=Y))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    # and the factor is applied: the data differ from the lossless ones
    d0 = orc.born_apply(g, R, T, A, f, dc)
    assert np.abs(orc.born_apply(g, R, T, A, f, dc, Lam=L, y=Y) - d0).max() > 1e-3 * np.abs(d0).max()


def test_zero_alpha_is_lossless(orc):
    """alpha0 = 0: Lam = 0 everywhere and the data equal the lossless ones."""
    g, c, tx, R = _homog(n=48, h=0.5, R=10.0, n_tx=5)
    K = P.born_fan_rays(R, g.h)
    T, A, L = orc.fan_maps(g, c, tx, R, 0.05, K, alpha0=np.zeros_like(c))
    assert (L == 0).all()
    dc = P.SplitMix64(2).normal(c.size).reshape(c.shape)
    f = P.born_frequencies(2)
    np.testing.assert_array_equal(orc.born_apply(g, R, T, A, f, dc, Lam=L, y=Y), orc.born_apply(g, R, T, A, f, dc))
