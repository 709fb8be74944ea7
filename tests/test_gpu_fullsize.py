"""Full-size GPU checks, in the launch configuration bench.py times.

Breast workload (1024^2 grid, 512-ring, 261,632 pairs) and the fish-eye lens
(512^2, 256-ring, 65,280 pairs): every pair is linked on the GPU; the oracle
checks a sample of pairs one by one, and properties that hold at any size
(dot-product identity, closed forms, finite differences) check the rest.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FAN = 256


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_18511_gb300 as m
    return m


@pytest.fixture(scope="module")
def P():
    from paper_2511_18511_gb300 import phantoms
    return phantoms


@pytest.fixture(scope="module")
def breast(P, rt):
    w = P.cfg_breast()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    return w, prob


def _np(t):
    return t.detach().cpu().numpy()


def _sample_pairs(P, n_tx, emitters, stride):
    pairs = P.all_pairs(n_tx)
    idx = np.flatnonzero(np.isin(pairs[:, 0], emitters))[::stride]
    return idx, pairs[idx]


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_breast_all_pairs_sampled_against_oracle(breast, orc, rt, P, prec):
    """All pairs linked on the GPU (cold, fan start); 4 emitters x every 4th
    receiver checked against the oracle pair by pair."""
    w, prob = breast
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == prob.n_pairs
    idx, sub = _sample_pairs(P, w.n_tx, [0, 131, 262, 393], 4)
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, pairs=sub, fan_rays=FAN)
    T = _np(r["tof"])[idx]
    hit = _np(r["hit"])[idx]
    rel = np.abs(T / ref["tof"] - 1)
    d_rx = np.linalg.norm(_np(r["hit"]) - w.tx[P.all_pairs(w.n_tx)[:, 1]], axis=1)
    print(f"[{prec}] breast full size: {len(idx)} sampled pairs, max ToF rel err {rel.max():.3e}, "
          f"max |hit - x_r| over all pairs {d_rx.max():.3e} mm, traces/pair {_np(r['iters']).mean():.3f}")
    assert rel.max() <= 2e-6
    assert d_rx.max() <= w.tol
    assert np.linalg.norm(hit - ref["hit"], axis=1).max() <= 2 * w.tol
    if prec == "fp64":
        np.testing.assert_array_equal(_np(r["iters"])[idx], ref["iters"])


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_breast_adjoint_dot_identity_and_sample(breast, orc, rt, P, prec):
    """<T(theta), w> = <s, L^T w> over all pairs (same rays on both sides of the
    identity), and the adjoint of a pair subset against the oracle's at the
    oracle's angles on the full grid."""
    w, prob = breast
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec)
    wt = torch.as_tensor(P.SplitMix64(41).normal(prob.n_pairs), device="cuda")
    T, _ = rt.rt_tof_forward(prob, r["theta"], w.ds, precision=prec)
    g = rt.rt_tof_adjoint(prob, r["theta"], wt, w.ds, precision=prec)
    lhs = float((T * wt).sum())
    rhs = float(-(g * prob.c).sum())          # <s, L^T w> with s = 1000/c, g = -1000 L^T w / c^2
    rel = abs(lhs - rhs) / float((T.abs() * wt.abs()).sum())
    print(f"[{prec}] dot identity rel {rel:.3e}")
    assert rel <= (1e-12 if prec == "fp64" else 2e-6)
    idx, sub = _sample_pairs(P, w.n_tx, [7, 300], 8)
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, pairs=sub, fan_rays=FAN)
    gw = P.SplitMix64(42).normal(len(sub))
    want = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"], gw, pairs=sub)
    prob_s = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius, pairs=sub)
    got = _np(rt.rt_tof_adjoint(prob_s, torch.as_tensor(ref["theta"], device="cuda"),
                                torch.as_tensor(gw, device="cuda"), w.ds, precision=prec))
    e_l2 = np.linalg.norm(got - want) / np.linalg.norm(want)
    e_max = np.abs(got - want).max() / np.abs(want).max()
    print(f"[{prec}] sampled adjoint on the full grid: rel L2 {e_l2:.3e}, rel max {e_max:.3e}")
    assert e_l2 <= 1e-5 and e_max <= 1e-5


def _fisheye_reference(tx, pairs, a=40.0, c0=1.5):
    xe, xr = tx[pairs[:, 0]], tx[pairs[:, 1]]
    chord = a * np.linalg.norm(xe - xr, axis=1) / np.sqrt((a * a + (xe ** 2).sum(1)) * (a * a + (xr ** 2).sum(1)))
    T = a * (2.0 * np.pi - 2.0 * np.arcsin(chord)) / c0
    # launch direction: tangent at e of the circle through e, its conjugate point and r,
    # oriented along the arc that passes the conjugate point first
    th = np.empty(len(pairs))
    for k in range(len(pairs)):
        e, r = xe[k], xr[k]
        cj = -(a * a / (e @ e)) * e
        A = np.array([[2 * (r - e)[0], 2 * (r - e)[1]], [2 * (cj - e)[0], 2 * (cj - e)[1]]])
        b = np.array([r @ r - e @ e, cj @ cj - e @ e])
        if abs(np.linalg.det(A)) < 1e-9 * np.abs(A).max() ** 2:
            th[k] = np.arctan2(*(r - e)[::-1])    # diametric pair: the ray is the straight diameter
            continue
        ctr = np.linalg.solve(A, b)
        t = np.array([-(e - ctr)[1], (e - ctr)[0]])
        # rotating from e towards the conjugate point must come before reaching r
        ang = lambda p: np.arctan2(*(p - ctr)[::-1])
        a_e, a_c, a_r = ang(e), ang(cj), ang(r)
        ccw_c = np.mod(a_c - a_e, 2 * np.pi) < np.mod(a_r - a_e, 2 * np.pi)
        th[k] = np.arctan2(*(t if ccw_c else -t)[::-1])
    return T, th


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_fisheye_full_size(orc, rt, P, prec):
    """Fish-eye lens at full size: ToF against the closed form (all pairs),
    launch angles against the analytic circles (sample), and the oracle on a
    sample of pairs."""
    w = P.cfg_fisheye()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec)
    ok, counts = rt.rt_status_counts()
    assert ok
    pairs = P.all_pairs(w.n_tx)
    xe, xr = w.tx[pairs[:, 0]], w.tx[pairs[:, 1]]
    a, c0 = 40.0, 1.5
    chord = a * np.linalg.norm(xe - xr, axis=1) / np.sqrt((a * a + (xe ** 2).sum(1)) * (a * a + (xr ** 2).sum(1)))
    T_true = a * (2.0 * np.pi - 2.0 * np.arcsin(chord)) / c0
    rel_true = np.abs(_np(r["tof"]) / T_true - 1)
    idx = np.arange(0, len(pairs), 97)
    _, th_true = _fisheye_reference(w.tx, pairs[idx])
    dth = np.abs(np.angle(np.exp(1j * (_np(r["theta"])[idx] - th_true))))
    sub_idx, sub = _sample_pairs(P, w.n_tx, [0, 85, 170], 5)
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, pairs=sub, fan_rays=FAN)
    rel_orc = np.abs(_np(r["tof"])[sub_idx] / ref["tof"] - 1)
    print(f"[{prec}] fish-eye 512^2/256-ring: ToF vs closed form max {rel_true.max():.3e} "
          f"(rms {np.sqrt(np.mean(rel_true ** 2)):.3e}); launch-angle deviation from the analytic "
          f"circles max {dth.max():.3e} rad (mean {dth.mean():.3e}); ToF vs oracle max {rel_orc.max():.3e}")
    assert rel_true.max() < 2e-5          # bilinear interpolation error at h = 0.2 mm
    assert dth.max() < 2e-4
    assert rel_orc.max() <= 2e-6


def test_breast_finite_differences_autograd(breast, rt, P):
    """Differentiable ToF (autograd backward = the adjoint kernel) against
    central differences with h = 0.01 m/s on 64 random pixels crossed by the
    rays, FP64 with tight relinking (FP32 cannot resolve the ~1e-9 us changes).
    A pixel whose perturbation moves some pair to another ray (a caustic: the
    travel time jumps) has no derivative there and is skipped, and counted."""
    w, prob_all = breast
    idx, sub = _sample_pairs(P, w.n_tx, np.arange(0, 512, 16), 16)    # 32 emitters x 32 receivers
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius, pairs=sub)
    tol = 1e-9
    c = prob.c.clone().requires_grad_(True)
    T = rt.tof(c, prob, w.ds, tol=tol, precision="fp64")
    wt = torch.as_tensor(P.SplitMix64(43).normal(len(sub)), device="cuda")
    (T * wt).sum().backward()
    g = _np(c.grad).ravel()
    base_r = rt.rt_link(prob, w.ds, tol=tol, precision="fp64")
    theta0 = base_r["theta"].clone()
    T0 = base_r["tof"].clone()
    x, y = w.grid.node_xy()
    inside = (x * x + y * y).ravel() < (0.8 * w.ring_radius) ** 2
    cand = np.flatnonzero(inside & (np.abs(g) > 0.05 * np.abs(g).max()))
    rng = P.SplitMix64(44)
    order = cand[(rng.uniform(4 * 64) * len(cand)).astype(int)]
    base = prob.c.clone()
    fd, ad, skipped = [], [], 0
    for j in order:
        if len(fd) == 64:
            break
        J, jump = [], 0.0
        for sgn in (1.0, -1.0):
            c2 = base.clone().view(-1)
            c2[j] += sgn * 0.01
            r2 = rt.rt_link(prob, w.ds, tol=tol, precision="fp64", theta0=theta0, c=c2.view_as(base))
            jump = max(jump, float((r2["tof"] - T0).abs().max()))
            J.append(float((r2["tof"] * wt).sum()))
        if jump > 1e-4:
            skipped += 1
            continue
        fd.append((J[0] - J[1]) / 0.02)
        ad.append(g[j])
    fd, ad = np.array(fd), np.array(ad)
    err = np.linalg.norm(fd - ad) / np.linalg.norm(ad)
    print(f"finite differences ({len(fd)} pixels, h = 0.01 m/s, {skipped} skipped at caustics): rel L2 {err:.3e}")
    assert len(fd) == 64 and skipped <= 16
    assert err <= 1e-2


def test_recorded_rows_breast(breast, rt):
    """The bench's step with recorded rows (rt_link_rows + rt_tof_adjoint_rows,
    cold fan of 768 rays at h/2) against rt_link + rt_tof_adjoint on the
    breast workload: identical links, every pair's row recorded, and the
    gradient equal up to the order of its FP64 sums."""
    w, prob = breast
    t_ref = rt.rt_link(prob, w.ds, tol=w.tol, precision="fp64", fan_rays=768)["tof"].clone() * 0.999
    sep = rt.rt_link(prob, w.ds, tol=w.tol, fan_rays=768, fan_ds=0.1)
    g_sep = rt.rt_tof_adjoint(prob, sep["theta"], sep["tof"], w.ds, tof_ref=t_ref)
    rows = rt.Rows.create(prob)
    out = rt.rt_link_rows(prob, w.ds, rows, tol=w.tol, fan_rays=768, fan_ds=0.1)
    g = rt.rt_tof_adjoint_rows(prob, rows, out["theta"], out["tof"], w.ds, tof_ref=t_ref)
    torch.cuda.synchronize()
    for k in ("theta", "tof", "hit", "status", "iters"):
        assert torch.equal(out[k], sep[k]), k
    ln = _np(rows.len)
    gs = _np(g_sep)
    rel = np.abs(_np(g) - gs).max() / np.abs(gs).max()
    print(f"breast recorded rows: runs per ray {ln.mean():.0f} (max {ln.max()}, cap {rows.cap}), "
          f"rows missing {(ln < 0).sum()}, gradient vs rt_tof_adjoint max rel {rel:.2e}")
    assert (ln > 0).all()
    assert rel <= 1e-11


def test_link_rounds_breast(breast, rt):
    """The bench's step linked in rounds with the R12 sub-fan (8 rays) on the
    breast workload against the single launch: every pair linked, the first
    two traces of every pair as in the single launch, travel times within the
    FP32 linking bar (the same rays), at most as many traces per pair on
    average, and the gradient from the recorded rows equal to the retracing
    adjoint at the linked angles."""
    w, prob = breast
    one = rt.rt_link(prob, w.ds, tol=w.tol, fan_rays=768, fan_ds=0.1)
    it1 = one["iters"].clone()
    rows = rt.Rows.create(prob)
    out = rt.rt_link_rows(prob, w.ds, rows, tol=w.tol, fan_rays=768, fan_ds=0.1, subfan_rays=8)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == prob.n_pairs
    it = out["iters"]
    early = it1 <= 2
    assert torch.equal(it[early], it1[early])
    rel = float((out["tof"] / one["tof"] - 1).abs().max())
    t_ref = out["tof"] * 0.999
    g = rt.rt_tof_adjoint_rows(prob, rows, out["theta"], out["tof"], w.ds, tof_ref=t_ref)
    g_tr = rt.rt_tof_adjoint(prob, out["theta"], out["tof"], w.ds, tof_ref=t_ref)
    grel = float((g - g_tr).abs().max() / g_tr.abs().max())
    h = torch.bincount(it.long()).tolist()
    h1 = torch.bincount(it1.long()).tolist()
    print(f"breast rounds with sub-fan: traces/pair {it.float().mean().item():.4f} {h} (single launch "
          f"{it1.float().mean().item():.4f} {h1}); ToF vs single launch max rel {rel:.2e}; "
          f"gradient rows vs retrace {grel:.2e}")
    assert rel <= 2e-6
    assert it.float().mean() <= it1.float().mean() + 1e-3
    assert (rows.len >= 0).all() and grel <= 1e-11
