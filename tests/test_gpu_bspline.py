"""The interpolating cubic B-spline sampler (paper Sec. 3.3.1, second scheme) on
the GPU against the oracle with the same sampler: the spline coefficients in
both directions, linking, travel times at the oracle's angles, endpoints, the
adjoint and the system matrix, both precisions and both integrators, on the
128^2 / 64-ring case; the paper's Sec. 4.2 acoustic-length experiment in its
own B-spline set-up; and the calls that refuse the option."""
import ctypes as C
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FAN = 256
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_18511_gb300 as m
    return m


@pytest.fixture(scope="module")
def case(rt, orc):
    from paper_2511_18511_gb300 import phantoms as P
    w = P.cfg_small()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    gw = P.SplitMix64(61).normal(prob.n_pairs)
    refs = {}
    for integ in ("rk4", "heun"):
        with orc.interpolator("bspline"), orc.integrator(integ):
            ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=FAN)
            adj = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"], gw)
            mat = orc.path_matrix(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"]) if integ == "rk4" else None
        refs[integ] = (ref, adj, mat)
    return w, prob, gw, refs


def _np(t):
    return t.detach().cpu().numpy()


def test_bspline_coefficients_match_oracle(case, rt, orc):
    w, prob, _, _ = case
    from paper_2511_18511_gb300 import phantoms as P
    for nx, ny in ((w.grid.nx, w.grid.ny), (37, 3), (3, 41), (50, 29)):
        g = P.Grid(nx, ny, 0.5)
        f = P.SplitMix64(nx * 100 + ny).normal(nx * ny).reshape(ny, nx)
        ft = torch.as_tensor(f, device="cuda")
        for tr in (False, True):
            a = _np(rt.bspline_coef(ft, transpose=tr))
            ref = orc.bspline_coef(g, f, transpose=tr)
            assert np.abs(a - ref).max() <= 1e-13 * np.abs(ref).max(), (nx, ny, tr)
    # in place
    f = torch.as_tensor(w.c / 1500.0, device="cuda")
    a = rt.bspline_coef(f, out=f)
    assert a.data_ptr() == f.data_ptr()
    assert np.abs(_np(a) - orc.bspline_coef(w.grid, w.c / 1500.0)).max() <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("integ", ["rk4", "heun"])
def test_bspline_link_tof_adjoint_match_oracle(case, rt, prec, integ):
    w, prob, gw, refs = case
    ref, adj, _ = refs[integ]
    assert (ref["status"] == 0).all()
    kw = dict(precision=prec, integrator=integ, interpolator="bspline")
    r = rt.rt_link(prob, w.ds, tol=w.tol, **kw)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == prob.n_pairs
    rel = np.abs(_np(r["tof"]) / ref["tof"] - 1).max()
    th = torch.as_tensor(ref["theta"], device="cuda")
    T, hit = rt.rt_tof_forward(prob, th, w.ds, **kw)
    rel_same = np.abs(_np(T) / ref["tof"] - 1).max()
    dend = np.linalg.norm(_np(hit) - ref["hit"], axis=1).max()
    g = _np(rt.rt_tof_adjoint(prob, th, torch.as_tensor(gw, device="cuda"), w.ds, **kw))
    e_adj = np.linalg.norm(g - adj) / np.linalg.norm(adj)
    print(f"[{prec} {integ} bspline] linked ToF {rel:.2e}, same-angle ToF {rel_same:.2e}, endpoint {dend:.2e} mm, "
          f"adjoint {e_adj:.2e}, traces/pair {_np(r['iters']).mean():.2f} (oracle {ref['iters'].mean():.2f})")
    if prec == "fp64":
        assert rel <= 1e-12 and rel_same <= 1e-12 and dend <= 1e-9 and e_adj <= 1e-10
        np.testing.assert_array_equal(_np(r["iters"]), ref["iters"])
    else:
        assert rel <= 2e-6 and rel_same <= 2e-6 and dend <= 1e-4 and e_adj <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_bspline_path_matrix_matches_oracle(case, rt, prec):
    """Rows over the slowness coefficients, entry for entry after summing
    duplicates, and T = L bspline_coef(s) through the library's own calls."""
    sp = pytest.importorskip("scipy.sparse")
    w, prob, _, refs = case
    ref, _, (rp, col, val) = refs["rk4"]
    n = w.grid.nx * w.grid.ny
    th = torch.as_tensor(ref["theta"], device="cuda")
    row_ptr, c_, v_ = rt.rt_path_matrix(prob, th, w.ds, precision=prec, interpolator="bspline")
    A = sp.csr_matrix((_np(v_), _np(c_), _np(row_ptr)), shape=(prob.n_pairs, n))
    B = sp.csr_matrix((val, col, rp), shape=(prob.n_pairs, n))
    D = (A - B).tocsr()
    err = np.abs(D.data).max() / np.abs(B.data).max() if D.nnz else 0.0
    # FP32: entries move with the trajectory (measured 3.9e-6 of the largest
    # entry; the bilinear rows measure 4.9e-6 under the same bar)
    assert err <= (1e-11 if prec == "fp64" else 1e-5), err
    s = torch.as_tensor(1000.0 / w.c, device="cuda")
    T = _np(rt.csr_matvec(row_ptr, c_, v_, rt.bspline_coef(s).reshape(-1)))
    assert np.abs(T / ref["tof"] - 1).max() <= (1e-12 if prec == "fp64" else 2e-6)


def test_bspline_differs_from_bilinear_and_bad_interpolator(case, rt):
    """The option reaches the kernels, and unknown samplers are refused."""
    w, prob, _, refs = case
    th = torch.as_tensor(refs["rk4"][0]["theta"], device="cuda")
    Tb, _ = rt.rt_tof_forward(prob, th, w.ds, precision="fp64", interpolator="bspline")
    Tl, _ = rt.rt_tof_forward(prob, th, w.ds, precision="fp64")
    assert float((Tb - Tl).abs().max()) > 1e-6
    with pytest.raises(ValueError):
        rt.rt_link(prob, w.ds, interpolator="nearest")
    L = rt._L.load()
    ps = prob.struct()
    theta = torch.full((prob.n_pairs,), float("nan"), dtype=torch.float64, device="cuda")
    o = rt._opts(w.ds)
    o.interpolator = 7
    assert L.rt_link(rt.default_context().h, C.byref(ps), C.byref(o), C.c_void_p(theta.data_ptr()), None, None,
                     None, None, None) == rt._L.RT_EINVAL
    # ray-Born maps take both samplers, not others (full-size outputs, so
    # nothing could be written out of bounds)
    o = rt._opts(w.ds)
    o.interpolator = 7
    T = torch.empty(prob.n_tx * w.grid.nx * w.grid.ny, dtype=torch.float32, device="cuda")
    A = torch.empty_like(T)
    assert L.rtborn_maps(rt.default_context().h, C.byref(ps), C.byref(o), 64, C.c_void_p(T.data_ptr()),
                         C.c_void_p(A.data_ptr()), None) == rt._L.RT_EINVAL


@pytest.mark.parametrize("integrator", ["rk4", "heun"])
def test_bspline_paper_acoustic_length_experiment_gpu(rt, orc, integrator):
    """Sec. 4.2 in the paper's own set-up: 2D fish-eye n = 1/(1 + r^2), a = 1,
    dx = 2 pi a/360, 101 rays from [0, a] to [0, -a] (L_true = a pi/2), with the
    cubic B-spline: per-ray parity with the oracle and the RE_al it gives."""
    from paper_2511_18511_gb300 import phantoms as P
    gold = json.load(open(os.path.join(GOLD, "fisheye_paper.json")))
    ex = gold["length_experiment"]
    h = gold["dx_over_a"] * gold["a"]
    n = 2 * int(np.ceil(1.15 / h)) + 1
    g = P.Grid(n, n, h)
    x, y = g.node_xy()
    c = 1000.0 * (1.0 + x * x + y * y)
    xp, xq = np.array(ex["x_p"]), np.array(ex["x_intercept"])
    axis = np.arctan2(*(np.array(ex["x_c"]) - xp)[::-1])
    thetas = axis + np.linspace(ex["theta_min"], ex["theta_max"], ex["n_rays"])
    pairs = np.tile(np.array([[0, 1]], np.int32), (len(thetas), 1))
    prob = rt.Problem.create(g, c, np.stack([xp, xq]), 1.0, pairs=pairs)
    th = torch.as_tensor(thetas, device="cuda")
    rows = []
    for ratio in (1.0, 0.5, 0.25):
        ds = ratio * h
        with orc.interpolator("bspline"), orc.integrator(integrator):
            L_o = np.array([orc.trace(g, c, 1.0, xp, xq, t, ds, record=False)["T"] for t in thetas])
        out = {"oracle": L_o}
        for prec in ("fp64", "fp32c"):
            T, _ = rt.rt_tof_forward(prob, th, ds, precision=prec, integrator=integrator, interpolator="bspline")
            out[prec] = _np(T)
            rel = np.abs(out[prec] / L_o - 1).max()
            assert rel <= (1e-12 if prec == "fp64" else 2e-6), (integrator, ratio, prec, rel)
        rows.append((ratio, *[100 * np.mean((out[k] - ex["L_true"]) / ex["L_true"]) for k in ("oracle", "fp64", "fp32c")]))
    print(f"\nRE_al (%) [{integrator}, B-spline], ds/dx: oracle / GPU FP64 / GPU FP32-comp")
    for r in rows:
        print(f"  {r[0]:6.3f}: {r[1]:+.4e} / {r[2]:+.4e} / {r[3]:+.4e}")
    assert all(abs(r[1]) < 1e-2 for r in rows)
