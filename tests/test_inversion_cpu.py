"""The inversion drivers' linear solvers (paper Sec. 3.1: SART, the default,
and conjugate gradients for each linearised subproblem) checked on CPU
against numpy on small seeded sparse systems: CG against the least-squares
solution (with and without damping), SART against the exact solution of a
consistent system and against its weighted fixed point."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")

from paper_2511_18511_gb300 import inversion as I


def _op(A):
    At = A.T.tocsr()
    return I.Operator(lambda x: torch.as_tensor(A @ x.numpy()), lambda w: torch.as_tensor(At @ w.numpy()),
                      A.shape[0], A.shape[1])


def _system(seed=1, m=300, n=80):
    A = sp.random(m, n, density=0.2, random_state=seed, format="csr")
    A.data = np.abs(A.data) + 0.1          # path lengths are non-negative
    return A


@pytest.mark.parametrize("damp", [0.0, 0.5])
def test_cg_reaches_least_squares(damp):
    A = _system()
    rng = np.random.default_rng(2)
    b = torch.as_tensor(rng.normal(size=A.shape[0]))
    x = I.cgls_solve(_op(A), b, 500, damp).numpy()
    Aa = np.vstack([A.toarray(), damp * np.eye(A.shape[1])])
    xl = np.linalg.lstsq(Aa, np.concatenate([b.numpy(), np.zeros(A.shape[1])]), rcond=None)[0]
    assert np.linalg.norm(x - xl) <= 1e-8 * np.linalg.norm(xl)


def test_sart_solves_consistent_system_and_keeps_bounds():
    A = _system(3)
    rng = np.random.default_rng(4)
    x_true = rng.uniform(0.6, 0.7, A.shape[1])
    b = torch.as_tensor(A @ x_true)
    x = I.sart_solve(_op(A), b, torch.full((A.shape[1],), 0.65, dtype=torch.float64), 2000).numpy()
    assert np.linalg.norm(x - x_true) <= 1e-10 * np.linalg.norm(x_true)
    xb = I.sart_solve(_op(A), b, torch.full((A.shape[1],), 0.65, dtype=torch.float64), 50,
                      lower=0.62, upper=0.68).numpy()
    assert xb.min() >= 0.62 and xb.max() <= 0.68


def test_sart_fixed_point_is_weighted_least_squares():
    """For an inconsistent system SART (relax 1) converges to the minimiser of
    ||R^-1/2 (A x - b)||^2 (Andersen and Kak's weighting)."""
    A = _system(5)
    rng = np.random.default_rng(6)
    b = torch.as_tensor(rng.uniform(20, 30, A.shape[0]))
    x = I.sart_solve(_op(A), b, torch.zeros(A.shape[1], dtype=torch.float64), 5000).numpy()
    w = 1.0 / np.sqrt(np.asarray(A.sum(axis=1)).ravel())
    xw = np.linalg.lstsq(A.toarray() * w[:, None], b.numpy() * w, rcond=None)[0]
    assert np.linalg.norm(x - xw) <= 1e-8 * np.linalg.norm(xw)


# ---------------------------------------------------------------- ray-Born

def test_complex_data_cg_reaches_least_squares():
    """min ||F x - b||^2 over real x, F complex: the CG iterate equals the
    solution of Re(F^H F) x = Re(F^H b) from numpy."""
    rng = np.random.default_rng(5)
    F = rng.normal(size=(120, 40)) + 1j * rng.normal(size=(120, 40))
    b = rng.normal(size=120) + 1j * rng.normal(size=120)
    Ft = torch.as_tensor(F)
    apply = lambda x: Ft @ x.to(torch.complex128)
    adjoint = lambda d: (Ft.conj().T @ d).real
    x = I.cg_complex_data(apply, adjoint, torch.as_tensor(b), torch.zeros(40, dtype=torch.float64), 200, rtol=1e-14)
    H = (F.conj().T @ F).real
    xl = np.linalg.solve(H, (F.conj().T @ b).real)
    assert np.linalg.norm(x.numpy() - xl) <= 1e-9 * np.linalg.norm(xl)


def _born_case(orc):
    from paper_2511_18511_gb300 import phantoms as P
    g = P.Grid(32, 32, 0.5)
    R = 7.0
    tx = P.ring(8, R)
    c = P.homogeneous(g, 1500.0)
    K = P.born_fan_rays(R, g.h)
    T, A = orc.fan_maps(g, c, tx, R, 0.05, K)
    x, y = g.node_xy()
    dc_true = 6.0 * np.exp(-((x - 1.5) ** 2 + (y + 1.0) ** 2) / 4.0) - 4.0 * np.exp(-((x + 2.0) ** 2 + y ** 2) / 2.0)
    dc_true[x * x + y * y >= R * R] = 0.0
    f = np.array([0.3, 0.45, 0.6, 0.75, 0.9, 1.05])
    d = orc.born_apply(g, R, T, A, f, dc_true)
    return g, R, T, A, f, d, dc_true


def oracle_born_ops(orc, g, R, T, A):
    apply = lambda f, x: torch.as_tensor(orc.born_apply(g, R, T, A, np.array(f), x.numpy()))
    adjoint = lambda f, d: torch.as_tensor(orc.born_adjoint(g, R, T, A, np.array(f), d.numpy()))
    return apply, adjoint


def test_born_frequency_marching_on_oracle_operators(orc):
    """Frequency marching (three levels of two frequencies, low to high) on
    consistent Born data of a smooth two-blob perturbation: each level lowers
    its own misfit by a large factor, the estimate approaches the truth, and
    the updates shrink from level to level."""
    g, R, T, A, f, d, dc_true = _born_case(orc)
    ops = oracle_born_ops(orc, g, R, T, A)
    res = I.born_frequency_marching(None, torch.as_tensor(d), f, [[0, 1], [2, 3], [4, 5]], n_inner=15,
                                    tol_update=0.0, dc0=torch.zeros(g.ny, g.nx, dtype=torch.float64), ops=ops)
    m = res.misfit
    assert res.levels_run == 3
    for k in range(3):
        assert m[2 * k + 1] <= 0.05 * m[2 * k], m
    err = np.linalg.norm(res.dc.numpy() - dc_true) / np.linalg.norm(dc_true)
    assert err < 0.6, err
    assert res.update[2] < res.update[0], res.update


def _born_case_strong(orc):
    """The 32^2 / 8-ring case with a contrast of tens of m/s, large enough that
    the Green's functions traced in the perturbed medium differ from the
    background's (travel-time shifts of a fraction of a period at 1 MHz)."""
    from paper_2511_18511_gb300 import phantoms as P
    g = P.Grid(32, 32, 0.5)
    R = 7.0
    tx = P.ring(8, R)
    c0 = P.homogeneous(g, 1500.0)
    K = P.born_fan_rays(R, g.h)
    x, y = g.node_xy()
    dc_true = 40.0 * np.exp(-((x - 1.5) ** 2 + (y + 1.0) ** 2) / 4.0) - 30.0 * np.exp(-((x + 2.0) ** 2 + y ** 2) / 2.0)
    dc_true[x * x + y * y >= R * R] = 0.0
    f = np.array([0.3, 0.45, 0.6, 0.75, 0.9, 1.05])

    def ops_in(dc):
        T, A = orc.fan_maps(g, c0 + np.asarray(dc, dtype=np.float64), tx, R, 0.05, K)
        return oracle_born_ops(orc, g, R, T, A)

    # Born data whose Green's functions are traced in the true medium
    d = ops_in(dc_true)[0](list(f), torch.as_tensor(dc_true)).numpy()
    return g, R, tx, c0, K, f, d, dc_true, ops_in


def test_ray_update_keeps_the_exact_estimate(orc):
    """Rays updated at every level (Sec. 3.1): started at the true perturbation
    with operators traced in the true medium, every level begins on a zero
    residual, which holds only if each rebuild traces in the background plus
    the current estimate (not the background, not the previous level's
    estimate) and the level's residual is d - F_k dc_k."""
    g, R, tx, c0, K, f, d, dc_true, ops_in = _born_case_strong(orc)
    levels = [[0, 1], [2, 3], [4, 5]]
    scale = 0.5 * float(np.sum(np.abs(d) ** 2))
    res = I.born_frequency_marching(None, torch.as_tensor(d), f, levels, n_inner=4, tol_update=0.0,
                                    dc0=torch.as_tensor(dc_true), ops=ops_in(dc_true), update_rays=ops_in)
    assert res.levels_run == 3
    for k in range(3):
        assert res.misfit[2 * k] <= 1e-20 * scale, res.misfit
    # on the background's operators the same start is far from a zero residual
    bg = I.born_frequency_marching(None, torch.as_tensor(d), f, levels, n_inner=4, tol_update=0.0,
                                   dc0=torch.as_tensor(dc_true), ops=ops_in(np.zeros_like(dc_true)))
    for k, lev in enumerate(levels):
        assert bg.misfit[2 * k] >= 1e-4 * 0.5 * float(np.sum(np.abs(d[lev]) ** 2)), bg.misfit


def test_ray_update_beats_fixed_background(orc):
    """On Born data whose Green's functions are traced in the true medium,
    marching from zero with the rays re-traced at every level ends nearer the
    truth than the same loop on the background's rays, and each level lowers
    its own misfit."""
    g, R, tx, c0, K, f, d, dc_true, ops_in = _born_case_strong(orc)
    levels = [[0, 1], [2, 3], [4, 5]]
    zero = torch.zeros(g.ny, g.nx, dtype=torch.float64)
    fixed = I.born_frequency_marching(None, torch.as_tensor(d), f, levels, n_inner=15, tol_update=0.0,
                                      dc0=zero, ops=ops_in(zero.numpy()))
    upd = I.born_frequency_marching(None, torch.as_tensor(d), f, levels, n_inner=15, tol_update=0.0,
                                    dc0=zero, ops=ops_in(zero.numpy()), update_rays=ops_in)
    e_fixed = np.linalg.norm(fixed.dc.numpy() - dc_true) / np.linalg.norm(dc_true)
    e_upd = np.linalg.norm(upd.dc.numpy() - dc_true) / np.linalg.norm(dc_true)
    print(f"model error: fixed background rays {e_fixed:.3f}, rays updated per level {e_upd:.3f}; "
          f"misfit {['%.2e' % m for m in upd.misfit]}")
    for k in range(3):
        assert upd.misfit[2 * k + 1] <= 0.1 * upd.misfit[2 * k], upd.misfit
    # the first level is the same solve on both
    assert abs(upd.misfit[1] - fixed.misfit[1]) <= 1e-9 * fixed.misfit[1]
    assert e_upd < e_fixed, (e_upd, e_fixed)
