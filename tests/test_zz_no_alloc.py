"""The allocation-free travel-time call (rt_tof_forward_noalloc).

It exists for callers that cannot allocate device memory when they need
travel times: its packed field lives in a fixed device array inside the
library instead of rt_ctx workspace. The test calls it through the C ABI
twice in a row and checks both results against rt_tof_forward at the same
angles, within the tolerances of the other parity tests. This file is
collected last so that a failure here leaves every other test already run.
"""
import ctypes as C

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


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_noalloc_matches_regular_call_twice(rt, orc, prec):
    from paper_2511_18511_gb300 import phantoms as P
    L = rt._L.load()
    w = P.cfg_small()
    ref = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, fan_rays=rt.DEFAULT_FAN)
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    theta = torch.as_tensor(ref["theta"], device="cuda")
    T_reg, hit_reg = rt.rt_tof_forward(prob, theta, w.ds, precision=prec)
    T_orc, _ = orc.tof(w.grid, w.c, w.tx, w.ring_radius, w.ds, ref["theta"])
    ps = prob.struct()
    o = rt._opts(w.ds, precision=prec)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        T = torch.full_like(T_reg, float("nan"))
        hit = torch.full_like(hit_reg, float("nan"))
        rc = L.rt_tof_forward_noalloc(C.byref(ps), C.byref(o), C.c_void_p(theta.data_ptr()),
                                      C.c_void_p(T.data_ptr()), C.c_void_p(hit.data_ptr()), stream)
        assert rc == rt._L.RT_OK
        torch.cuda.synchronize()
        rel = (T / T_reg - 1).abs().max().item()
        assert rel <= (1e-12 if prec == "fp64" else 2e-6), rel
        assert (hit - hit_reg).abs().max().item() <= (1e-9 if prec == "fp64" else 1e-4)
        # and, independently of the regular call, against the oracle at the same angles
        rel_o = np.abs(T.cpu().numpy() / T_orc - 1).max()
        assert rel_o <= (1e-12 if prec == "fp64" else 2e-6), rel_o


def test_noalloc_rejects_grids_beyond_its_scratch(rt):
    from paper_2511_18511_gb300 import phantoms as P
    L = rt._L.load()
    g = P.Grid(1024, 1024, 0.2)          # 1023^2 cells x 64 B > 16 MiB
    prob = rt.Problem.create(g, P.homogeneous(g), P.ring(8, 95.0), 95.0)
    ps = prob.struct()
    o = rt._opts(0.02, precision="fp32c")
    theta = torch.zeros(prob.n_pairs, dtype=torch.float64, device="cuda")
    T = torch.full_like(theta, float("nan"))
    torch.cuda.synchronize()
    rc = L.rt_tof_forward_noalloc(C.byref(ps), C.byref(o), C.c_void_p(theta.data_ptr()),
                                  C.c_void_p(T.data_ptr()), None, None)
    assert rc == rt._L.RT_ENOMEM
    torch.cuda.synchronize()
    assert torch.isnan(T).all()          # nothing was enqueued: the output is untouched
