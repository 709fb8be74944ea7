"""Pins of reading R13, an option of the oracle's fan-started linking: the
second and third angles come from the fan's interpolating polynomial moved
onto the linking traces (an offset through the first trace, then an offset
and a tilt through the first two), instead of R8's inverse quartic and secant.

The closed-form pins give the fan rays on a polynomial and the traces on that
polynomial moved by a known offset and tilt: the predicted angle must be the
moved polynomial's root. The workload pin runs both rules on eight emitters of
the breast workload that hold its longest linking chains."""
import numpy as np
import pytest

from paper_2511_18511_gb300 import phantoms as P


def _cubic(c, tc):
    return lambda t: c[0] + c[1] * (t - tc) + c[2] * (t - tc) ** 2 + c[3] * (t - tc) ** 3


def _root_in(coef_desc, lo, hi):
    r = np.roots(coef_desc)
    r = r[np.abs(r.imag) < 1e-12].real
    r = r[(r > lo) & (r < hi)]
    assert r.size == 1
    return float(r[0])


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("n", [8, 4])
def test_r13_angle_exact_for_moved_cubic(orc, sign, n):
    """Fan rays on a cubic p (both orientations), traces on p + a0 (one trace)
    or p + a0 + b0 (theta - x1) (two traces): the angle is the root of the moved
    cubic, to rounding."""
    tc, c = 0.135, (0.0, 20.0, 300.0, 2000.0)
    t = 0.135 + 0.01 * (np.arange(n) - (n - 1) / 2)
    p = _cubic(c, tc)
    m = sign * p(t)
    lo, hi = 0.13, 0.14
    a0, b0, x1, x2 = 0.03, 3.0, 0.137, 0.131
    # one trace: f = s p + a0
    th = orc.r13_angle(t, m, x1, sign * p(x1) + a0, lo, hi)
    u_desc = [sign * c[3], sign * c[2], sign * c[1], sign * c[0] + a0]          # in u = theta - tc
    exact = tc + _root_in(u_desc, lo - tc, hi - tc)
    assert abs(th - exact) <= 1e-12, (th, exact)
    # two traces: f = s p + a0 + b0 (theta - x1)
    f = lambda x: sign * p(x) + a0 + b0 * (x - x1)
    th2 = orc.r13_angle(t, m, x1, f(x1), lo, hi, x2=x2, m2=f(x2))
    u_desc2 = [sign * c[3], sign * c[2], sign * c[1] + b0, sign * c[0] + a0 + b0 * (tc - x1)]
    exact2 = tc + _root_in(u_desc2, lo - tc, hi - tc)
    assert abs(th2 - exact2) <= 1e-12, (th2, exact2)
    assert abs(f(th2)) <= 1e-12


def test_r13_angle_linear_window_and_no_sign_change(orc):
    """Two fan rays: the model is their chord moved onto the trace, so a
    misfit that is that chord plus an offset is solved exactly; a moved model
    without a sign change over the interval gives NaN (the R8 rule then picks
    the angle)."""
    t = np.array([1.0, 1.01])
    m = np.array([-0.2, 0.3])                      # slope 50
    th = orc.r13_angle(t, m, 1.004, -0.2 + 50 * 0.004 + 0.05, 1.0, 1.01)
    assert abs(th - (1.0 + (0.2 - 0.05) / 50)) <= 1e-14
    assert np.isnan(orc.r13_angle(t, m, 1.004, 5.0, 1.0, 1.01))


def test_r13_links_the_same_rays_in_fewer_traces(orc):
    """Eight emitters of the breast workload (1024^2, 512-ring, 768-ray fan at
    0.1 mm) that hold its longest linking chains: with R13 every pair still
    links, to the same rays as R8 (ToF within 1e-8), a pair that links in one
    trace is untouched, the pairs needing three or more traces fall to at most
    a third and the longest chain is shorter (R8: 56 pairs at >= 3 traces, up
    to 6; R13: 11, up to 5)."""
    w = P.cfg_breast()
    em = [189, 190, 202, 217, 289, 303, 317, 336]
    pairs = np.array([(e, r) for e in em for r in range(w.n_tx) if r != e], np.int32)
    kw = dict(tol=w.tol, fan_rays=768, fan_ds=0.1, pairs=pairs)
    a = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, **kw)
    with orc.link_rule("r13"):
        b = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, **kw)
    c = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, **kw)      # the rule is restored
    np.testing.assert_array_equal(c["iters"], a["iters"])
    assert (a["status"] == 0).all() and (b["status"] == 0).all()
    np.testing.assert_allclose(b["tof"], a["tof"], rtol=1e-8)
    one = a["iters"] == 1
    np.testing.assert_array_equal(b["iters"] == 1, one)
    np.testing.assert_array_equal(b["theta"][one], a["theta"][one])
    n3a, n3b = int((a["iters"] >= 3).sum()), int((b["iters"] >= 3).sum())
    assert n3a >= 40 and n3b <= n3a / 3, (np.bincount(a["iters"]), np.bincount(b["iters"]))
    assert b["iters"].max() < a["iters"].max()
    assert b["iters"].sum() < a["iters"].sum()
