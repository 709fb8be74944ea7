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
