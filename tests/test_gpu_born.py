"""Ray-Born on the GPU (rtborn_maps / rtborn_apply / rtborn_adjoint) against
the FP64 oracle: fan maps on the scaled-down instance (128^2, 64-ring), the
Born map and its adjoint on seeded synthetic maps (the same float32 values on
both sides), the whole chain maps -> data, the dot-product identity, autograd,
and sampled checks at full size (1024^2, 512-ring, 8 frequencies)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def small(rt, P, orc):
    w = P.cfg_born_small()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    maps = rt.rtborn_maps(prob, w.ds, w.fan_rays)
    T_o, A_o = orc.fan_maps(w.grid, w.c, w.tx, w.ring_radius, w.ds, w.fan_rays)
    return w, prob, maps, T_o, A_o


def _synthetic_maps(P, grid, tx, seed):
    """Seeded float32 maps: straight-ray times at 1.5 mm/us plus a ripple,
    amplitude 1/sqrt(r); one unreached node per map."""
    x, y = grid.node_xy()
    rng = P.SplitMix64(seed)
    T = np.empty((len(tx), grid.ny, grid.nx), np.float32)
    A = np.empty_like(T)
    for t in range(len(tx)):
        r = np.hypot(x - tx[t, 0], y - tx[t, 1]) + 0.1
        T[t] = r / 1.5 + 0.05 * rng.normal(x.size).reshape(x.shape)
        A[t] = 1.0 / np.sqrt(r)
        T[t, 5 + t % 7, 9] = np.inf
        A[t, 5 + t % 7, 9] = 0.0
    return T, A


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------- fan maps

def test_maps_small_vs_oracle(small, P):
    """FP32 maps against the FP64 oracle's: every node inside the ring reached
    on both sides; travel times within 2e-6 of the largest; amplitudes (of the
    candidate of least T + eta (b/h)^2) within 1e-4 relative at 99.9% of the
    nodes. The rest are nodes where two candidates' scores lie within the FP32
    rounding of T, which the two precisions order differently."""
    w, prob, maps, T_o, A_o = small
    T, A = _np(maps.T), _np(maps.A)
    x, y = w.grid.node_xy()
    inside = x * x + y * y < (w.ring_radius - 2 * w.grid.h) ** 2
    assert np.isfinite(T[:, inside]).all() and np.isfinite(T_o[:, inside]).all()
    relT = np.abs(T[:, inside] / T_o[:, inside] - 1)
    absT = np.abs(T[:, inside] - T_o[:, inside])
    relA = np.abs(A[:, inside] / A_o[:, inside] - 1)
    q = np.quantile(relA, [0.5, 0.99, 0.999])
    print(f"maps 128^2/64-ring vs oracle: T rel max {relT.max():.2e} (abs {absT.max():.2e} us), "
          f"A rel median {q[0]:.2e} p99 {q[1]:.2e} p99.9 {q[2]:.2e} max {relA.max():.2e}, "
          f"fraction > 1e-3: {(relA > 1e-3).mean():.2e}")
    assert absT.max() <= 2e-6 * T_o[:, inside].max()
    assert q[2] <= 1e-4 and (relA > 1e-3).mean() <= 1e-3
    outside = x * x + y * y > (w.ring_radius + 2 * w.grid.h) ** 2
    assert np.isinf(T[:, outside]).all() and (A[:, outside] == 0).all()


# --------------------------------------------------------- Born map, adjoint

@pytest.mark.parametrize("grad,tol_t,tol_a", [(1.0, 2e-6, 5e-5), (5.0, 2e-5, 1.5e-4)])
def test_maps_linear_gradient_closed_form_gpu(rt, P, grad, tol_t, tol_a):
    """The GPU fan maps in c = 1500 + grad y against the closed forms of the
    circular rays (travel time, and amplitude from Q = |x - x_e| / |cos a|):
    within the oracle's bounds plus the FP32 rounding of T (a few 1e-7) and A."""
    from tests.test_oracle_born_pins import linear_gradient_maps_closed_form
    g = P.Grid(64, 64, 0.5)
    R = 14.0
    tx = P.ring(8, R)
    prob = rt.Problem.create(g, P.linear_gradient(g, 1500.0, grad), tx, R)
    maps = rt.rtborn_maps(prob, 0.05, P.born_fan_rays(R, g.h))
    T, A = _np(maps.T), _np(maps.A)
    x, y = g.node_xy()
    inside = x * x + y * y < R * R
    worst_t = worst_a = 0.0
    for t in range(len(tx)):
        Tc, Ac, r, adx = linear_gradient_maps_closed_form(g, grad, tx[t])
        m = inside & (r >= 2 * g.h) & (adx > 2 * g.h)
        worst_t = max(worst_t, float(np.abs(T[t][m] / Tc[m] - 1).max()))
        worst_a = max(worst_a, float(np.abs(A[t][m] / Ac[m] - 1).max()))
    print(f"linear gradient {grad} (m/s)/mm, GPU maps vs closed form: T rel max {worst_t:.2e}, A rel max {worst_a:.2e}")
    assert worst_t <= tol_t + 1e-6 and worst_a <= tol_a + 1e-5


@pytest.mark.parametrize("gemm", ["fp32", "tf32x3"])
def test_apply_adjoint_synthetic_maps_vs_oracle(rt, P, orc, gemm):
    """Born map and adjoint of the same float32 maps on both sides (128^2,
    64-ring, 8 frequencies): complex64 data within 1e-4 relative L2 of the
    oracle, the adjoint too."""
    w = P.cfg_born_small()
    T, A = _synthetic_maps(P, w.grid, w.tx, 21)
    maps = rt.BornMaps(w.grid, w.ring_radius, torch.as_tensor(T, device="cuda"), torch.as_tensor(A, device="cuda"))
    dc = w.dc.astype(np.float32)
    d = _np(rt.rtborn_apply(maps, w.f_mhz, torch.as_tensor(dc, device="cuda"), gemm=gemm))
    want = orc.born_apply(w.grid, w.ring_radius, T.astype(np.float64), A.astype(np.float64), w.f_mhz,
                          dc.astype(np.float64))
    e_apply = _rel_l2(d, want)
    rng = P.SplitMix64(22)
    n = len(w.f_mhz) * w.n_tx * w.n_tx
    dd = (rng.normal(n) + 1j * rng.normal(n)).reshape(len(w.f_mhz), w.n_tx, w.n_tx).astype(np.complex64)
    g = _np(rt.rtborn_adjoint(maps, w.f_mhz, torch.as_tensor(dd, device="cuda"), gemm=gemm))
    want_g = orc.born_adjoint(w.grid, w.ring_radius, T.astype(np.float64), A.astype(np.float64), w.f_mhz,
                              dd.astype(np.complex128))
    e_adj = _rel_l2(g, want_g)
    print(f"[{gemm}] apply rel L2 {e_apply:.2e} (max {np.abs(d - want).max() / np.abs(want).max():.2e}), "
          f"adjoint rel L2 {e_adj:.2e}")
    assert np.all(np.abs(d[:, np.arange(w.n_tx), np.arange(w.n_tx)]) == 0)
    assert e_apply <= 1e-4 and e_adj <= 1e-4


def _predicted_error(T, A, T_o, A_o, f_mhz, mask, dc=None, pairs=None):
    """Relative L2 error of the Born data (dc given) or adjoint (dc None) that
    the maps' own FP32 error implies. Per node the product E_e E_r carries
    the relative error delta = dA_e/A_e + dA_r/A_r + i omega (dT_e + dT_r); for
    an i.i.d. zero-mean perturbation (or data) the expected squared relative
    error of the sums is the mean of |delta|^2 weighted by |omega^2 A_e A_r dc|^2
    (or |omega^2 A_e A_r|^2) over the nodes and pairs summed."""
    n = T.shape[0]
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b] if pairs is None else pairs
    num = den = 0.0
    for f in f_mhz:
        om = 2 * np.pi * f
        for a, b in pairs:
            m = mask & np.isfinite(T_o[a]) & np.isfinite(T_o[b]) & (A_o[a] > 0) & (A_o[b] > 0)
            dl = (A[a][m] / A_o[a][m] - 1) + (A[b][m] / A_o[b][m] - 1) + \
                1j * om * ((T[a][m] - T_o[a][m]) + (T[b][m] - T_o[b][m]))
            wgt = (om ** 2 * A_o[a][m] * A_o[b][m] * (1.0 if dc is None else dc[m])) ** 2
            num += float(np.sum(wgt * np.abs(dl) ** 2))
            den += float(np.sum(wgt))
    return float(np.sqrt(num / den))


def test_chain_maps_apply_vs_oracle(small, rt, orc):
    """GPU maps -> GPU data against oracle maps -> oracle data (128^2,
    64-ring): within the 1e-4 relative L2 of the scope's sampled-apply bar, and
    within twice the error that the FP32 maps' own error implies (phase
    omega dT and amplitude; _predicted_error) plus the contraction's 1e-5."""
    w, prob, maps, T_o, A_o = small
    dc = w.dc.astype(np.float32)
    d = _np(rt.rtborn_apply(maps, w.f_mhz, torch.as_tensor(dc, device="cuda"), gemm="fp32"))
    want = orc.born_apply(w.grid, w.ring_radius, T_o, A_o, w.f_mhz, dc.astype(np.float64))
    e = _rel_l2(d, want)
    per_f = [_rel_l2(d[k], want[k]) for k in range(len(w.f_mhz))]
    x, y = w.grid.node_xy()
    inside = x * x + y * y < w.ring_radius ** 2
    pred = _predicted_error(_np(maps.T).astype(np.float64), _np(maps.A).astype(np.float64), T_o, A_o, w.f_mhz,
                            inside, dc=dc.astype(np.float64), pairs=[(a, (a + 17) % w.n_tx) for a in range(w.n_tx)])
    print(f"chain maps->data vs oracle: rel L2 {e:.2e} (predicted from the map errors {pred:.2e}); per frequency "
          + " ".join(f"{v:.1e}" for v in per_f))
    assert e <= 1e-4
    assert e <= 2 * pred + 1e-5


@pytest.mark.parametrize("gemm", ["fp32", "tf32x3"])
def test_dot_product_identity_gpu(small, rt, P, gemm):
    """Re<F dc, d> = <dc, F* d> through the GPU calls (maps from the GPU)."""
    w, prob, maps, _, _ = small
    rng = P.SplitMix64(23)
    dc = torch.as_tensor(rng.normal(w.grid.nx * w.grid.ny).reshape(w.grid.ny, w.grid.nx), dtype=torch.float32,
                         device="cuda")
    n = len(w.f_mhz) * w.n_tx * w.n_tx
    d = torch.as_tensor((rng.normal(n) + 1j * rng.normal(n)).reshape(len(w.f_mhz), w.n_tx, w.n_tx),
                        dtype=torch.complex64, device="cuda")
    Fd = rt.rtborn_apply(maps, w.f_mhz, dc, gemm=gemm)
    Fad = rt.rtborn_adjoint(maps, w.f_mhz, d, gemm=gemm)
    lhs = float((torch.conj(Fd).to(torch.complex128) * d.to(torch.complex128)).real.sum())
    rhs = float((dc.double() * Fad.double()).sum())
    scale = float((Fd.abs().double() * d.abs().double()).sum())
    print(f"[{gemm}] dot identity: {lhs:.6e} vs {rhs:.6e}, rel {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_born_autograd_backward_is_adjoint(rt, P, orc):
    """d = born(dc): backward of L = Re sum conj(w) d gives Re(F^H w), checked
    against the oracle's adjoint on the same synthetic maps."""
    w = P.cfg_born_small()
    T, A = _synthetic_maps(P, w.grid, w.tx, 24)
    maps = rt.BornMaps(w.grid, w.ring_radius, torch.as_tensor(T, device="cuda"), torch.as_tensor(A, device="cuda"))
    f = w.f_mhz[:3]
    dc = torch.as_tensor(w.dc, dtype=torch.float32, device="cuda").requires_grad_(True)
    rng = P.SplitMix64(25)
    n = len(f) * w.n_tx * w.n_tx
    wt = (rng.normal(n) + 1j * rng.normal(n)).reshape(len(f), w.n_tx, w.n_tx)
    d = rt.born(dc, maps, f, gemm="fp32")
    L = (torch.conj(torch.as_tensor(wt, dtype=torch.complex64, device="cuda")) * d).real.sum()
    L.backward()
    want = orc.born_adjoint(w.grid, w.ring_radius, T.astype(np.float64), A.astype(np.float64), f, wt)
    e = _rel_l2(_np(dc.grad), want)
    print(f"autograd backward vs oracle adjoint: rel L2 {e:.2e}")
    assert e <= 1e-4


def test_born_bad_arguments(rt, P, small):
    w, prob, maps, _, _ = small
    with pytest.raises(rt._L.RtError):
        rt.rtborn_maps(prob, w.ds, 1)
    with pytest.raises(rt._L.RtError):
        rt.rtborn_maps(prob, 2.0 * w.grid.h, 64)
    with pytest.raises(ValueError):
        rt.rtborn_apply(maps, w.f_mhz, torch.zeros(7, device="cuda"))
    L = rt._L.load()
    ctx = rt.default_context()
    g = maps._grid_struct()
    import ctypes as C
    fa = (C.c_double * 1)(1.0)
    rc = L.rtborn_apply(ctx.h, C.byref(g), maps.ring_radius, maps.n_tx, C.c_void_p(maps.T.data_ptr()),
                        C.c_void_p(maps.A.data_ptr()), 1, fa, C.c_void_p(maps.T.data_ptr()), 7,
                        C.c_void_p(maps.T.data_ptr()), None)
    assert rc == rt._L.RT_EINVAL


# ---------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def full(rt, P, orc):
    w = P.cfg_born()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    maps = rt.rtborn_maps(prob, w.ds, w.fan_rays)
    sel = np.array([0, 131, 262, 393])
    T_o, A_o = orc.fan_maps(w.grid, w.c, w.tx[sel], w.ring_radius, w.ds, w.fan_rays)
    return w, prob, maps, sel, T_o, A_o


def _near(mask, r):
    """Nodes within r nodes (Chebyshev) of a True node, per map."""
    out = mask.copy()
    n0, n1 = mask.shape[-2:]
    for dj in range(-r, r + 1):
        for di in range(-r, r + 1):
            out[..., max(dj, 0):n0 + min(dj, 0), max(di, 0):n1 + min(di, 0)] |= \
                mask[..., max(-dj, 0):n0 + min(-dj, 0), max(-di, 0):n1 + min(-di, 0)]
    return out


def test_full_size_maps_sampled(full):
    """1024^2, 512-ring, K = 6016: the maps of 4 transducers against the
    oracle's. Travel times within 1e-6 relative away from caustics. Within 3
    nodes of a caustic (a node whose |Q| < 2h, where the oracle's amplitude is
    near its clamp) the second-order term P/Q magnifies the FP32 error of Q,
    and the bound there is 2e-5 relative."""
    w, prob, maps, sel, T_o, A_o = full
    T, A = _np(maps.T[sel]), _np(maps.A[sel])
    x, y = w.grid.node_xy()
    inside = np.broadcast_to(x * x + y * y < (w.ring_radius - 2 * w.grid.h) ** 2, T.shape)
    reached = np.isfinite(T_o) & inside
    assert (np.isfinite(T[inside]) == reached[inside]).mean() > 0.9999
    both = reached & np.isfinite(T)
    caustic = _near(reached & (1.0 / np.maximum(A_o, 1e-30) ** 2 < 2.0 * w.grid.h), 3)
    calm = both & ~caustic
    rel_calm = np.abs(T[calm] / T_o[calm] - 1)
    rel_caus = np.abs(T[both & caustic] / T_o[both & caustic] - 1)
    relA = np.abs(A[calm] / A_o[calm] - 1)
    q = np.quantile(relA, [0.5, 0.99, 0.999])
    print(f"full-size maps (4 transducers): reached {both[inside].mean():.6f}, nodes near caustics "
          f"{(both & caustic).sum()}; T rel max {rel_calm.max():.2e} (near caustics {rel_caus.max():.2e}); "
          f"A rel median {q[0]:.2e} p99 {q[1]:.2e} p99.9 {q[2]:.2e} max {relA.max():.2e}")
    assert rel_calm.max() <= 1e-6 and rel_caus.max() <= 2e-5
    assert q[2] <= 1e-4 and (relA > 1e-3).mean() <= 1e-3


def _ambiguous(A_o, h, ratio=1.2):
    """Caustic zones, where which ray a node takes its amplitude from is
    decided by rounding on either side: nodes within 3 of a node whose oracle
    |Q| < 2h (amplitude near its clamp), or whose oracle amplitude varies by
    more than `ratio` within their 3 x 3 neighbourhood, in any of the maps."""
    hi = np.where(np.isfinite(A_o), A_o, 0.0)
    lo = np.where(hi > 0, hi, np.inf)
    mx, mn = hi.copy(), lo.copy()
    n0, n1 = hi.shape[-2:]
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            dst = (..., slice(max(dj, 0), n0 + min(dj, 0)), slice(max(di, 0), n1 + min(di, 0)))
            src = (..., slice(max(-dj, 0), n0 + min(-dj, 0)), slice(max(-di, 0), n1 + min(-di, 0)))
            mx[dst] = np.maximum(mx[dst], hi[src])
            mn[dst] = np.minimum(mn[dst], lo[src])
    caustic = _near(np.isfinite(A_o) & (1.0 / np.maximum(A_o, 1e-30) ** 2 < 2.0 * h), 3)
    return ((mx > ratio * mn) | caustic).any(axis=0)


def test_full_size_apply_adjoint_sampled(full, rt, P, orc):
    """Full apply (8 frequencies, all 512 transducers) sampled at the pairs
    among the 4 oracle-mapped transducers, with the perturbation restricted to
    nodes away from caustic zones (where the amplitude choice is ambiguous; the
    unrestricted figure is printed and bounded loosely); the adjoint of data on
    those pairs against the oracle at the same nodes; the dot-product identity
    at full size."""
    w, prob, maps, sel, T_o, A_o = full
    amb = _ambiguous(A_o, w.grid.h)
    dcm = np.where(amb, 0.0, w.dc).astype(np.float32)
    d_all = rt.rtborn_apply(maps, w.f_mhz, torch.as_tensor(w.dc, dtype=torch.float32, device="cuda"), gemm="tf32x3")
    want_all = orc.born_apply(w.grid, w.ring_radius, T_o, A_o, w.f_mhz, w.dc.astype(np.float32).astype(np.float64))
    e_all = _rel_l2(_np(d_all)[:, sel][:, :, sel], want_all)
    d = rt.rtborn_apply(maps, w.f_mhz, torch.as_tensor(dcm, device="cuda"), gemm="tf32x3")
    want = orc.born_apply(w.grid, w.ring_radius, T_o, A_o, w.f_mhz, dcm.astype(np.float64))
    e = _rel_l2(_np(d)[:, sel][:, :, sel], want)
    x, y = w.grid.node_xy()
    inside = x * x + y * y < w.ring_radius ** 2
    Tg, Ag = _np(maps.T[sel]).astype(np.float64), _np(maps.A[sel]).astype(np.float64)
    pred = _predicted_error(Tg, Ag, T_o, A_o, w.f_mhz, inside & ~amb, dc=dcm.astype(np.float64))
    pred_all = _predicted_error(Tg, Ag, T_o, A_o, w.f_mhz, inside, dc=w.dc.astype(np.float64))
    print(f"full-size apply at the oracle-mapped pairs: rel L2 {e:.2e} away from caustic zones "
          f"({amb.sum()} nodes excluded; predicted from the map errors {pred:.2e}), {e_all:.2e} with them "
          f"(predicted {pred_all:.2e})")
    # the maps' FP32 error sets the data's: bounded by twice its prediction
    # plus the contraction's own error (1e-5), with and without caustic zones
    assert e <= 2 * pred + 1e-5 and e_all <= 2 * pred_all + 1e-5
    rng = P.SplitMix64(26)
    n = len(w.f_mhz) * len(sel) ** 2
    ds_ = (rng.normal(n) + 1j * rng.normal(n)).reshape(len(w.f_mhz), len(sel), len(sel))
    full_d = torch.zeros((len(w.f_mhz), w.n_tx, w.n_tx), dtype=torch.complex64, device="cuda")
    idx = torch.as_tensor(sel, device="cuda")
    full_d[:, idx[:, None], idx[None, :]] = torch.as_tensor(ds_, dtype=torch.complex64, device="cuda")
    g = _np(rt.rtborn_adjoint(maps, w.f_mhz, full_d, gemm="tf32x3"))
    want_g = orc.born_adjoint(w.grid, w.ring_radius, T_o, A_o, w.f_mhz, ds_)
    e_g = _rel_l2(np.where(amb, 0, g), np.where(amb, 0, want_g))
    pred_g = _predicted_error(Tg, Ag, T_o, A_o, w.f_mhz, inside & ~amb)
    print(f"full-size adjoint of data on the oracle-mapped pairs: rel L2 {e_g:.2e} away from caustic zones "
          f"(predicted from the map errors {pred_g:.2e})")
    assert e_g <= 2 * pred_g + 1e-5
    dc = torch.as_tensor(w.dc, dtype=torch.float32, device="cuda")
    dd = torch.as_tensor((rng.normal(len(w.f_mhz) * w.n_tx ** 2) + 1j * rng.normal(len(w.f_mhz) * w.n_tx ** 2))
                         .reshape(len(w.f_mhz), w.n_tx, w.n_tx), dtype=torch.complex64, device="cuda")
    Fad = rt.rtborn_adjoint(maps, w.f_mhz, dd, gemm="tf32x3")
    lhs = float((torch.conj(d_all).to(torch.complex128) * dd.to(torch.complex128)).real.sum())
    rhs = float((dc.double() * Fad.double()).sum())
    scale = float((d_all.abs().double() * dd.abs().double()).sum())
    print(f"full-size dot identity rel {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-5 * scale
