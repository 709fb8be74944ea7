"""Travel-time inversion on the GPU (paper Sec. 3.1): the CSR products with the
system matrix against scipy, and a few SART / CG linearisations on the
128^2 / 64-ring Gaussian-inclusion phantom from a homogeneous start."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")

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
def case(rt):
    from paper_2511_18511_gb300 import phantoms as P
    w = P.cfg_small()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    meas = rt.rt_link(prob, w.ds, tol=1e-6, precision="fp64")
    return w, prob, meas["tof"].clone(), meas["theta"].clone()


def test_csr_products_match_scipy(case, rt):
    w, prob, _, theta = case
    row_ptr, col, val = rt.rt_path_matrix(prob, theta, w.ds, precision="fp64")
    n = w.grid.nx * w.grid.ny
    A = sp.csr_matrix((val.cpu().numpy(), col.cpu().numpy(), row_ptr.cpu().numpy()), shape=(prob.n_pairs, n))
    rng = np.random.default_rng(7)
    x = rng.normal(size=n)
    wv = rng.normal(size=prob.n_pairs)
    y = rt.csr_matvec(row_ptr, col, val, torch.as_tensor(x, device="cuda")).cpu().numpy()
    z = rt.csr_rmatvec(row_ptr, col, val, torch.as_tensor(wv, device="cuda"), n).cpu().numpy()
    assert np.abs(y - A @ x).max() <= 1e-12 * np.abs(A @ x).max()
    assert np.abs(z - A.T @ wv).max() <= 1e-12 * np.abs(A.T @ wv).max()
    # T = L s at the linked rays (the matrix rows are the travel-time weights)
    T = rt.csr_matvec(row_ptr, col, val, (1000.0 / prob.c).reshape(-1))
    assert float((T - case[2]).abs().max()) <= 1e-10 * float(case[2].max())


@pytest.mark.parametrize("solver", ["sart", "cg"])
def test_inversion_reduces_misfit_and_model_error(case, rt, solver):
    from paper_2511_18511_gb300 import inversion as I
    w, prob, t_meas, _ = case
    c0 = torch.full_like(prob.c, 1500.0)
    res = I.invert_tof(prob, t_meas, w.ds, n_lin=4, n_inner=20, solver=solver, c0=c0, damp=0.0)
    c_true = prob.c
    x, y = w.grid.node_xy()
    inside = torch.as_tensor(x * x + y * y < (0.8 * w.ring_radius) ** 2, device="cuda")
    e0 = float((c0 - c_true)[inside].norm() / (c_true[inside] - 1500.0).norm())
    e1 = float((res.c - c_true)[inside].norm() / (c_true[inside] - 1500.0).norm())
    print(f"[{solver}] misfit per linearisation {['%.3e' % m for m in res.misfit]}, traces {res.traces}, "
          f"model error {e0:.3f} -> {e1:.3f}")
    assert res.misfit[-1] <= 0.1 * res.misfit[0]
    assert all(b <= a * 1.05 for a, b in zip(res.misfit, res.misfit[1:]))
    assert e1 <= 0.8 * e0


# ---------------------------------------------------------------- ray-Born frequency marching

def test_born_marching_gpu_matches_oracle_loop(rt, orc):
    """The marching loop over the GPU Born operators against the same loop over
    the FP64 oracle operators, on the same (oracle) maps: every level lowers
    its misfit by a large factor on both, and the estimates agree."""
    from tests.test_inversion_cpu import _born_case, oracle_born_ops
    from paper_2511_18511_gb300 import inversion as I
    g, R, T, A, f, d, dc_true = _born_case(orc)
    levels = [[0, 1], [2, 3], [4, 5]]
    ref = I.born_frequency_marching(None, torch.as_tensor(d), f, levels, n_inner=15, tol_update=0.0,
                                    dc0=torch.zeros(g.ny, g.nx, dtype=torch.float64),
                                    ops=oracle_born_ops(orc, g, R, T, A))
    maps = rt.BornMaps(g, R, torch.as_tensor(T, dtype=torch.float32, device="cuda"),
                       torch.as_tensor(A, dtype=torch.float32, device="cuda"))
    res = I.born_frequency_marching(maps, torch.as_tensor(d, dtype=torch.complex64, device="cuda"), f, levels,
                                    n_inner=15, tol_update=0.0, gemm="fp32")
    e_gpu = float(np.linalg.norm(res.dc.cpu().numpy() - dc_true) / np.linalg.norm(dc_true))
    e_ref = float(np.linalg.norm(ref.dc.numpy() - dc_true) / np.linalg.norm(dc_true))
    diff = float(np.linalg.norm(res.dc.cpu().numpy() - ref.dc.numpy()) / np.linalg.norm(ref.dc.numpy()))
    print(f"Born marching: misfit GPU {['%.2e' % m for m in res.misfit]}, oracle {['%.2e' % m for m in ref.misfit]}; "
          f"model error GPU {e_gpu:.3f} oracle {e_ref:.3f}; estimates differ by {diff:.2e}")
    for k in range(3):
        assert res.misfit[2 * k + 1] <= 0.05 * res.misfit[2 * k]
    assert abs(e_gpu - e_ref) <= 0.02 and diff <= 0.05


def test_born_marching_ray_update_gpu_matches_oracle_loop(rt, orc):
    """The marching loop with the rays re-traced in the background plus the
    current estimate at every level (Sec. 3.1), on GPU maps and operators,
    against the same loop on the FP64 oracle's maps and operators, on Born data
    whose Green's functions are traced in the true medium (contrast of tens of
    m/s): every level lowers its misfit on both, both end nearer the truth than
    the loop on the background's rays, and the estimates agree."""
    from tests.test_inversion_cpu import _born_case_strong
    from paper_2511_18511_gb300 import inversion as I
    g, R, tx, c0, K, f, d, dc_true, ops_in = _born_case_strong(orc)
    levels = [[0, 1], [2, 3], [4, 5]]
    zero = torch.zeros(g.ny, g.nx, dtype=torch.float64)
    ref = I.born_frequency_marching(None, torch.as_tensor(d), f, levels, n_inner=15, tol_update=0.0,
                                    dc0=zero, ops=ops_in(zero.numpy()), update_rays=ops_in)
    fixed = I.born_frequency_marching(None, torch.as_tensor(d), f, levels, n_inner=15, tol_update=0.0,
                                      dc0=zero, ops=ops_in(zero.numpy()))
    prob = rt.Problem.create(g, c0, tx, R)
    update = I.gpu_ray_update(prob, 0.05, K, gemm="fp32")
    dc0 = torch.zeros(g.ny, g.nx, dtype=torch.float32, device="cuda")
    res = I.born_frequency_marching(None, torch.as_tensor(d, dtype=torch.complex64, device="cuda"), f, levels,
                                    n_inner=15, tol_update=0.0, dc0=dc0, ops=update(dc0), update_rays=update)
    out = res.dc.cpu().double().numpy()
    e_gpu = float(np.linalg.norm(out - dc_true) / np.linalg.norm(dc_true))
    e_ref = float(np.linalg.norm(ref.dc.numpy() - dc_true) / np.linalg.norm(dc_true))
    e_fix = float(np.linalg.norm(fixed.dc.numpy() - dc_true) / np.linalg.norm(dc_true))
    diff = float(np.linalg.norm(out - ref.dc.numpy()) / np.linalg.norm(ref.dc.numpy()))
    print(f"Born marching with ray update: misfit GPU {['%.2e' % m for m in res.misfit]}, oracle "
          f"{['%.2e' % m for m in ref.misfit]}; model error GPU {e_gpu:.3f} oracle {e_ref:.3f} "
          f"(background rays {e_fix:.3f}); estimates differ by {diff:.2e}")
    for k in range(3):
        assert res.misfit[2 * k + 1] <= 0.1 * res.misfit[2 * k]
    assert e_gpu < e_fix and abs(e_gpu - e_ref) <= 0.02 and diff <= 0.05


def test_born_marching_on_gpu_maps(rt):
    """The loop at the scaled-down ray-Born size (128^2, 64-ring, 8 frequencies
    in four levels) on GPU maps: consistent data of a smooth perturbation."""
    from paper_2511_18511_gb300 import inversion as I
    from paper_2511_18511_gb300 import phantoms as P
    w = P.cfg_born_small()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    maps = rt.rtborn_maps(prob, w.ds, w.fan_rays)
    x, y = w.grid.node_xy()
    dc_true = 8.0 * np.exp(-((x - 6.0) ** 2 + (y + 4.0) ** 2) / 18.0) - 5.0 * np.exp(-((x + 8.0) ** 2 + (y - 5.0) ** 2) / 8.0)
    dc_true[x * x + y * y >= w.ring_radius ** 2] = 0.0
    dct = torch.as_tensor(dc_true, dtype=torch.float32, device="cuda")
    d = rt.rtborn_apply(maps, w.f_mhz, dct, gemm="fp32")
    res = I.born_frequency_marching(maps, d, w.f_mhz, [[0, 1], [2, 3], [4, 5], [6, 7]], n_inner=10,
                                    tol_update=0.0, gemm="fp32")
    err = float((res.dc - dct).norm() / dct.norm())
    print(f"Born marching 128^2/64-ring: misfit {['%.2e' % m for m in res.misfit]}, updates "
          f"{['%.2e' % u for u in res.update]}, model error {err:.3f}")
    for k in range(4):
        assert res.misfit[2 * k + 1] <= 0.1 * res.misfit[2 * k]
    assert err < 0.7
