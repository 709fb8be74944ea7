"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances of the ray path: travel time 2e-6 relative per pair, endpoints
1e-4 mm, adjoint 1e-5 relative (L2 and max-abs over the grid). Both the FP64
form (measured ~1e-14) and the FP32-compensated form (~1e-7 travel time,
~1e-6 adjoint) meet them. Linked endpoints are compared with the receiver
(tol) and with the oracle's linked endpoint within 2 tol, since each side stops
at its own iterate within tol of the receiver; rays traced from the same
angles are compared within 1e-4 mm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOF_RTOL = 2e-6
END_TOL = 1e-4
ADJ_RTOL = 1e-5


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


def _np(t):
    return t.detach().cpu().numpy()


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


FAN = 256   # the library's default cold start; fan 0 = the paper's straight-line start


@pytest.fixture(scope="module")
def small(orc, P, rt):
    w = P.cfg_small()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=FAN)
    return w, prob, ref


@pytest.fixture(scope="module")
def small_straight(orc, small):
    w, prob, _ = small
    return orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=0)


@pytest.mark.parametrize("fan", [FAN, 0])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_link_matches_oracle_small(small, small_straight, rt, P, prec, fan):
    """128^2 grid, 64-ring (4032 pairs, 32 blocks of 128 with a ragged tail),
    fan-predicted and straight-line cold starts."""
    w, prob, ref = small
    if fan == 0:
        ref = small_straight
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec, fan_rays=fan)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == prob.n_pairs
    st = _np(r["status"])
    assert (st == 0).all()
    rel = np.abs(_np(r["tof"]) / ref["tof"] - 1)
    assert rel.max() <= TOF_RTOL, rel.max()
    pairs = P.all_pairs(w.n_tx)
    hit = _np(r["hit"])
    # linking contract: every endpoint within tol of its receiver, on the ring
    d_rx = np.linalg.norm(hit - w.tx[pairs[:, 1]], axis=1).max()
    assert d_rx <= w.tol
    # on the ring to the position resolution (FP32: 6e-8 of a cell)
    np.testing.assert_allclose(np.linalg.norm(hit, axis=1), w.ring_radius,
                               rtol=1e-10 if prec == "fp64" else 3e-9)
    # each side stops at its own iterate within tol of the receiver, so the two
    # linked endpoints can differ by up to 2 tol; rays traced from the same
    # angles are held to END_TOL in test_tof_at_oracle_angles
    d_or = np.linalg.norm(hit - ref["hit"], axis=1)
    assert d_or.max() <= 2 * w.tol
    print(f"[{prec} fan={fan}] linked: max ToF rel err {rel.max():.3e}, max |hit - x_r| {d_rx:.3e} mm, "
          f"max |hit - hit_oracle| {d_or.max():.3e} mm (median {np.median(d_or):.3e}), "
          f"traces/pair {_np(r['iters']).mean():.2f} (oracle {ref['iters'].mean():.2f})")
    if prec == "fp64":
        np.testing.assert_array_equal(_np(r["iters"]), ref["iters"])


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_link_with_coarse_fan_matches_oracle(rt, orc, P, prec):
    """The fan start traced at its own step (fan_ds = h/2 = 5 ds, launch
    angles still following ds) against the oracle with the same fan step:
    every pair links, travel times and endpoints within the linking bars, and
    in FP64 the same number of traces per pair as the oracle."""
    w = P.cfg_small()
    fds = 0.5 * w.grid.h
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=FAN, fan_ds=fds)
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec, fan_rays=FAN, fan_ds=fds)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == prob.n_pairs
    rel = np.abs(_np(r["tof"]) / ref["tof"] - 1)
    assert rel.max() <= TOF_RTOL, rel.max()
    pairs = P.all_pairs(w.n_tx)
    assert np.linalg.norm(_np(r["hit"]) - w.tx[pairs[:, 1]], axis=1).max() <= w.tol
    it, it_ref = _np(r["iters"]), ref["iters"]
    print(f"[{prec} fan_ds={fds}] linked: max ToF rel err {rel.max():.3e}, traces/pair {it.mean():.4f} "
          f"(oracle {it_ref.mean():.4f}; fan at ds: oracle "
          f"{orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=FAN)['iters'].mean():.4f})")
    if prec == "fp64":
        np.testing.assert_array_equal(it, it_ref)
    else:
        assert abs(it.mean() - it_ref.mean()) <= 0.01


@pytest.mark.parametrize("subfan", [8, 16])
def test_link_rounds_with_subfan_match_oracle(rt, orc, P, subfan):
    """R12 on the GPU: the link in rounds (one trace per pair, the second
    traces, the sub-fan, the rest) with a coarse 16-ray fan, so that many
    pairs reach a third trace, against the oracle with the same sub-fan: every
    pair links, ToF and endpoints within the linking bars, the traces per pair
    as the oracle's (FP32 may move a few pairs by one trace); against the GPU's
    single launch without the sub-fan, the same rays and the same first two
    traces; with recorded rows, the same link and an adjoint from the rows that
    equals the retracing adjoint at the linked angles."""
    w = P.cfg_small()
    kw = dict(tol=w.tol, fan_rays=16, fan_ds=0.5 * w.grid.h)
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, subfan=subfan, **kw)
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    r = rt.rt_link(prob, w.ds, subfan_rays=subfan, **kw)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == prob.n_pairs
    rel = np.abs(_np(r["tof"]) / ref["tof"] - 1)
    assert rel.max() <= TOF_RTOL, rel.max()
    pairs = P.all_pairs(w.n_tx)
    assert np.linalg.norm(_np(r["hit"]) - w.tx[pairs[:, 1]], axis=1).max() <= w.tol
    it, it_ref = _np(r["iters"]), ref["iters"]
    assert (it >= 3).sum() > 1000
    same = np.mean(it == it_ref)
    print(f"[subfan {subfan}] GPU rounds vs oracle: max ToF rel err {rel.max():.3e}; traces/pair {it.mean():.4f} "
          f"(oracle {it_ref.mean():.4f}), same trace count on {same:.4f} of the pairs; histogram {np.bincount(it)}")
    assert same >= 0.99 and abs(it.mean() - it_ref.mean()) <= 0.01
    one = rt.rt_link(prob, w.ds, **kw)
    it1 = _np(one["iters"])
    early = it1 <= 2
    np.testing.assert_array_equal(it[early], it1[early])
    assert np.abs(_np(r["tof"]) / _np(one["tof"]) - 1).max() <= TOF_RTOL
    rows = rt.Rows.create(prob)
    rr = rt.rt_link_rows(prob, w.ds, rows, subfan_rays=subfan, **kw)
    for k in ("theta", "tof", "iters", "status"):
        assert torch.equal(rr[k], r[k]), k
    g_ref = torch.as_tensor(P.SplitMix64(5).normal(prob.n_pairs), device="cuda")
    g_rows = rt.rt_tof_adjoint_rows(prob, rows, rr["theta"], rr["tof"], w.ds, tof_ref=g_ref)
    g_tr = rt.rt_tof_adjoint(prob, rr["theta"], rr["tof"], w.ds, tof_ref=g_ref)
    assert (rows.len >= 0).all()
    assert float((g_rows - g_tr).abs().max() / g_tr.abs().max()) <= 1e-11
    with pytest.raises(rt._L.RtError):
        rt.rt_link(prob, w.ds, precision="fp64", subfan_rays=subfan, **kw)


@pytest.mark.parametrize("fan", [FAN, 0])
def test_recorded_rows_small(rt, orc, P, fan):
    """rt_link_rows links exactly as rt_link and records the linked rays' rows;
    rt_tof_adjoint_rows from them equals rt_tof_adjoint up to the order of the
    FP64 sums and the oracle's adjoint within the adjoint bar; with a cap of 8
    runs all but the shortest rows overflow and those pairs are traced again,
    with the same gradient (128^2 / 64-ring, fan and straight starts)."""
    w = P.cfg_small()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    g_ref = torch.as_tensor(P.SplitMix64(5).normal(prob.n_pairs), device="cuda")
    sep = rt.rt_link(prob, w.ds, tol=w.tol, fan_rays=fan)
    g_sep = rt.rt_tof_adjoint(prob, sep["theta"], sep["tof"], w.ds, tof_ref=g_ref)
    rows = rt.Rows.create(prob)
    out = rt.rt_link_rows(prob, w.ds, rows, tol=w.tol, fan_rays=fan)
    g = rt.rt_tof_adjoint_rows(prob, rows, out["theta"], out["tof"], w.ds, tof_ref=g_ref)
    torch.cuda.synchronize()
    for k in ("theta", "tof", "status", "iters"):
        assert torch.equal(out[k], sep[k]), k
    ln = _np(rows.len)
    assert (ln > 0).all() and ln.max() <= rows.cap
    ref = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, _np(out["theta"]), _np(out["tof"]) - _np(g_ref))
    gf, gs = _np(g), _np(g_sep)
    rel = np.linalg.norm(gf - ref) / np.linalg.norm(ref)
    same = np.abs(gf - gs).max() / np.abs(gs).max()
    tiny = rt.Rows.create(prob, cap=8)
    out2 = rt.rt_link_rows(prob, w.ds, tiny, tol=w.tol, fan_rays=fan)
    g2 = rt.rt_tof_adjoint_rows(prob, tiny, out2["theta"], out2["tof"], w.ds, tof_ref=g_ref)
    torch.cuda.synchronize()
    ln2 = _np(tiny.len)
    assert ((ln2 == -1) | ((ln2 >= 1) & (ln2 <= 8))).all() and (ln2 == -1).mean() > 0.9
    same2 = np.abs(_np(g2) - gs).max() / np.abs(gs).max()
    print(f"[fan={fan}] recorded rows: runs per ray {ln.mean():.0f} (max {ln.max()}, cap {rows.cap}), adjoint vs "
          f"oracle rel L2 {rel:.2e}, vs rt_tof_adjoint {same:.2e}, {(ln2 == -1).mean():.3f} of the rows "
          f"overflowing a cap of 8: {same2:.2e}")
    assert rel <= ADJ_RTOL and same <= 1e-11 and same2 <= 1e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_tof_at_oracle_angles(small, rt, prec):
    """Travel time at the oracle's linked angles (same rays on both sides)."""
    w, prob, ref = small
    th = torch.as_tensor(ref["theta"], device="cuda")
    T, hit = rt.rt_tof_forward(prob, th, w.ds, precision=prec)
    rel = np.abs(_np(T) / ref["tof"] - 1).max()
    bound = 1e-11 if prec == "fp64" else TOF_RTOL
    assert rel <= bound, rel
    endb = 1e-9 if prec == "fp64" else END_TOL
    dend = np.linalg.norm(_np(hit) - ref["hit"], axis=1).max()
    assert dend <= endb
    print(f"[{prec}] same angles: max ToF rel err {rel:.3e}, max endpoint diff {dend:.3e} mm")


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_adjoint_at_oracle_angles(small, orc, rt, P, prec):
    """Adjoint scatter at the oracle's angles against the oracle's L^T g."""
    w, prob, ref = small
    g = P.SplitMix64(5).normal(prob.n_pairs)
    want = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"], g)
    got = _np(rt.rt_tof_adjoint(prob, torch.as_tensor(ref["theta"], device="cuda"),
                                torch.as_tensor(g, device="cuda"), w.ds, precision=prec))
    e_l2 = _rel_l2(got, want)
    e_max = np.abs(got - want).max() / np.abs(want).max()
    bound = 1e-11 if prec == "fp64" else ADJ_RTOL
    print(f"[{prec}] adjoint at oracle angles: rel L2 {e_l2:.3e}, rel max {e_max:.3e}")
    assert e_l2 <= bound and e_max <= bound, (e_l2, e_max)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_full_pipeline_adjoint(small, orc, rt, P, prec):
    """Link + adjoint end to end (each side with its own linked rays). FP64
    reaches the same iterates as the oracle (measured ~1e-13); the FP32 form
    with compensated position and direction measured 8.5e-7 L2 / 1.2e-6 max."""
    w, prob, ref = small
    g = P.SplitMix64(6).normal(prob.n_pairs)
    want = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"], g)
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec)
    got = _np(rt.rt_tof_adjoint(prob, r["theta"], torch.as_tensor(g, device="cuda"), w.ds, precision=prec))
    e_l2 = _rel_l2(got, want)
    e_max = np.abs(got - want).max() / np.abs(want).max()
    print(f"[{prec}] adjoint end to end: rel L2 {e_l2:.3e}, rel max {e_max:.3e}")
    assert e_l2 <= ADJ_RTOL and e_max <= ADJ_RTOL, (e_l2, e_max)


def test_residual_weights_and_autograd(small, orc, rt, P):
    """tof_ref path (w = T - T_ref) and the autograd Function call the same kernel."""
    w, prob, ref = small
    c = prob.c.clone().requires_grad_(True)
    T = rt.tof(c, prob, w.ds, precision="fp64")
    Tref = T.detach() * 0.999
    loss = 0.5 * ((T - Tref) ** 2).sum()
    loss.backward()
    theta = torch.as_tensor(ref["theta"], device="cuda")
    g2 = rt.rt_tof_adjoint(prob, theta, T.detach(), w.ds, tof_ref=Tref, precision="fp64")
    want = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"], _np(T - Tref))
    assert _rel_l2(_np(c.grad), want) <= ADJ_RTOL
    assert _rel_l2(_np(g2), want) <= ADJ_RTOL


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_path_matrix_matches_oracle(small, orc, rt, prec):
    w, prob, ref = small
    sub = slice(0, 400)
    pairs = np.array([[e, r] for e in range(w.n_tx) for r in range(w.n_tx) if e != r], np.int32)[sub]
    prob2 = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius, pairs=pairs)
    th = ref["theta"][sub]
    rp, col, val = rt.rt_path_matrix(prob2, torch.as_tensor(th, device="cuda"), w.ds, precision=prec)
    orp, ocol, oval = orc.path_matrix(w.grid, w.c, w.tx, w.ring_radius, w.ds, th, pairs=pairs)
    import scipy.sparse as sp
    n = w.grid.nx * w.grid.ny
    A = sp.csr_matrix((_np(val), _np(col), _np(rp)), shape=(len(th), n)).toarray()
    B = sp.csr_matrix((oval, ocol, orp), shape=(len(th), n)).toarray()
    err = np.abs(A - B).max() / np.abs(B).max()
    print(f"[{prec}] path matrix at oracle angles: max entry error / max entry {err:.3e}")
    # FP32: entries move with the trajectory (measured 4.9e-6 of the largest entry)
    assert err <= (1e-11 if prec == "fp64" else 1e-5), err


def test_closed_forms_on_gpu(rt, P):
    """Homogeneous (T = chord/c) and linear-gradient (arccosh) closed forms."""
    g = P.Grid(128, 128, 0.5)
    tx = P.ring(64, 30.0)
    pairs = P.all_pairs(64)
    chord = np.linalg.norm(tx[pairs[:, 0]] - tx[pairs[:, 1]], axis=1)
    for prec in ("fp64", "fp32c"):
        prob = rt.Problem.create(g, P.homogeneous(g), tx, 30.0)
        r = rt.rt_link(prob, 0.05, precision=prec)
        assert np.abs(_np(r["tof"]) / (chord / 1.5) - 1).max() < (1e-12 if prec == "fp64" else 1e-6)
        prob = rt.Problem.create(g, P.linear_gradient(g, 1500.0, 1.0), tx, 30.0)
        r = rt.rt_link(prob, 0.05, tol=1e-6, precision=prec)
        xe, xr = tx[pairs[:, 0]], tx[pairs[:, 1]]
        ce, cr = 1.5 + 1e-3 * xe[:, 1], 1.5 + 1e-3 * xr[:, 1]
        T = np.arccosh(1 + 1e-6 * chord ** 2 / (2 * ce * cr)) / 1e-3
        # oracle: 2.7e-8 (slowness interpolation); FP32 adds its ~1.6e-7 travel-time error
        assert np.abs(_np(r["tof"]) / T - 1).max() < (5e-8 if prec == "fp64" else 4e-7)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_fisheye_against_oracle_and_closed_form(orc, rt, P, prec):
    """Strong refraction (fish-eye lens, 256^2 at 0.4 mm, 32-ring at 45 mm)."""
    w = P.cfg_fisheye(n=256, n_tx=32, h=0.4, ds=0.04)
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=FAN)
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec)
    assert (_np(r["status"]) == 0).all()
    rel = np.abs(_np(r["tof"]) / ref["tof"] - 1).max()
    assert rel <= TOF_RTOL, rel
    pairs = P.all_pairs(w.n_tx)
    assert np.linalg.norm(_np(r["hit"]) - w.tx[pairs[:, 1]], axis=1).max() <= w.tol
    d_or = np.linalg.norm(_np(r["hit"]) - ref["hit"], axis=1).max()
    assert d_or <= 2 * w.tol
    print(f"[{prec}] fish-eye: max ToF rel err {rel:.3e}, max |hit - hit_oracle| {d_or:.3e} mm")


def test_edge_cases(rt, P):
    import ctypes
    g = P.Grid(64, 64, 0.5)
    tx = P.ring(8, 14.0)
    c = P.homogeneous(g)
    # empty explicit pair list
    prob = rt.Problem.create(g, c, tx, 14.0, pairs=np.zeros((0, 2), np.int32))
    r = rt.rt_link(prob, 0.05)
    assert r["tof"].numel() == 0
    # ragged explicit list with an invalid pair (e == r) and an out-of-range index
    pairs = np.array([[0, 3], [2, 2], [1, 9], [5, 1]] * 33 + [[0, 1]], np.int32)
    prob = rt.Problem.create(g, c, tx, 14.0, pairs=pairs)
    r = rt.rt_link(prob, 0.05)
    st = _np(r["status"])
    assert (st[1::4][:33] == 4).all() and (st[2::4][:33] == 4).all() and st[0] == 0 and st[-1] == 0
    assert np.isnan(_np(r["tof"])[1])
    # bad sound speed -> every pair BADINPUT, no fault
    bad = c.copy()
    bad[10, 10] = -5.0
    prob = rt.Problem.create(g, bad, tx, 14.0)
    r = rt.rt_link(prob, 0.05)
    assert (_np(r["status"]) == 4).all()
    ok, counts = rt.rt_status_counts()
    assert not ok and counts[4] == prob.n_pairs
    # ring outside the grid -> RT_EINVAL before any launch
    prob = rt.Problem.create(g, c, P.ring(8, 20.0), 20.0)
    with pytest.raises(rt._L.RtError) as ei:
        rt.rt_link(prob, 0.05)
    assert ei.value.code == rt._L.RT_EINVAL
    # max_iter = 2 in a refracting medium leaves unconverged pairs, reported
    w = P.cfg_fisheye(n=256, n_tx=16, h=0.4, ds=0.04)
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    r = rt.rt_link(prob, w.ds, tol=1e-6, max_iter=2, fan_rays=0)
    ok, counts = rt.rt_status_counts()
    assert not ok and counts[1] > 0 and (_np(r["iters"]) <= 2).all()
    # warm start from linked angles: one trace per pair
    r2 = rt.rt_link(prob, w.ds, tol=1e-4)
    r3 = rt.rt_link(prob, w.ds, tol=1e-4, theta0=r2["theta"])
    assert (_np(r3["iters"]) == 1).all()
