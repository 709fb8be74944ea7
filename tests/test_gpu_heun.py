"""Heun's second-order Runge-Kutta stepper (the paper's default, Sec. 3.2.3)
on the GPU against the oracle traced with the same stepper: linking, travel
times at the oracle's angles, endpoints and the adjoint, both precisions, on
the 128^2 / 64-ring case."""
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
def case(rt, orc):
    from paper_2511_18511_gb300 import phantoms as P
    w = P.cfg_small()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    with orc.integrator("heun"):
        ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=FAN)
        gw = P.SplitMix64(51).normal(prob.n_pairs)
        adj = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"], gw)
    return w, prob, ref, gw, adj


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_heun_link_tof_adjoint_match_oracle(case, rt, prec):
    w, prob, ref, gw, adj = case
    assert (ref["status"] == 0).all()
    r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec, integrator="heun")
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == prob.n_pairs
    rel = np.abs(_np(r["tof"]) / ref["tof"] - 1).max()
    th = torch.as_tensor(ref["theta"], device="cuda")
    T, hit = rt.rt_tof_forward(prob, th, w.ds, precision=prec, integrator="heun")
    rel_same = np.abs(_np(T) / ref["tof"] - 1).max()
    dend = np.linalg.norm(_np(hit) - ref["hit"], axis=1).max()
    g = _np(rt.rt_tof_adjoint(prob, th, torch.as_tensor(gw, device="cuda"), w.ds, precision=prec,
                              integrator="heun"))
    e_adj = np.linalg.norm(g - adj) / np.linalg.norm(adj)
    print(f"[{prec} heun] linked ToF {rel:.2e}, same-angle ToF {rel_same:.2e}, endpoint {dend:.2e} mm, "
          f"adjoint {e_adj:.2e}, traces/pair {_np(r['iters']).mean():.2f} (oracle {ref['iters'].mean():.2f})")
    if prec == "fp64":
        assert rel <= 1e-12 and rel_same <= 1e-12 and dend <= 1e-9 and e_adj <= 1e-10
        np.testing.assert_array_equal(_np(r["iters"]), ref["iters"])
    else:
        assert rel <= 2e-6 and rel_same <= 2e-6 and dend <= 1e-4 and e_adj <= 1e-5


def test_heun_differs_from_rk4_and_bad_integrator(case, rt):
    """The option reaches the kernels (Heun's O(ds^2) path error is visible
    against RK4 at ds = 0.05 mm), and unknown integrators are refused."""
    w, prob, ref, _, _ = case
    th = torch.as_tensor(ref["theta"], device="cuda")
    Th, _ = rt.rt_tof_forward(prob, th, w.ds, precision="fp64", integrator="heun")
    Tr, _ = rt.rt_tof_forward(prob, th, w.ds, precision="fp64", integrator="rk4")
    assert float((Th - Tr).abs().max()) > 0
    with pytest.raises(ValueError):
        rt.rt_link(prob, w.ds, integrator="euler")
    import ctypes as C
    ps = prob.struct()
    o = rt._opts(w.ds)
    o.integrator = 7
    theta = torch.full((prob.n_pairs,), float("nan"), dtype=torch.float64, device="cuda")
    L = rt._L.load()
    assert L.rt_link(rt.default_context().h, C.byref(ps), C.byref(o), C.c_void_p(theta.data_ptr()), None, None,
                     None, None, None) == rt._L.RT_EINVAL
