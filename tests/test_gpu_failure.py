"""Failure detection without a GPU fault: the bounded wait that every pipeline
barrier of the tensor-core Born kernels uses gives up after its limit, records
its error code and returns; the context stays usable afterwards."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_18511_gb300 as rt
    return rt


def test_bounded_wait_completes_when_the_phase_does(rt):
    code, secs = rt.wait_selftest(50_000_000, arrive=True)
    assert code == 0 and secs < 1.0, (code, secs)


@pytest.mark.parametrize("limit_ms", [5, 40])
def test_bounded_wait_gives_up_and_reports(rt, limit_ms):
    """A barrier that nothing completes: the wait returns after its limit with
    the error code, the kernel ends, and the launch reports no CUDA error."""
    code, secs = rt.wait_selftest(limit_ms * 1_000_000, arrive=False)
    print(f"wait of {limit_ms} ms on a barrier nobody completes: code {code}, {secs * 1e3:.1f} ms wall")
    assert code == 199
    assert limit_ms * 1e-3 <= secs < limit_ms * 1e-3 + 1.0
    torch.cuda.synchronize()


def test_context_usable_after_a_wait_gave_up(rt, orc):
    """After a wait that gave up, the tensor-core Born apply still runs and
    matches the oracle on a small case."""
    from paper_2511_18511_gb300 import phantoms as P
    assert rt.wait_selftest(5_000_000, arrive=False)[0] == 199
    g = P.Grid(32, 32, 0.5)
    R, tx = 7.0, P.ring(8, 7.0)
    c = P.homogeneous(g, 1500.0)
    K = P.born_fan_rays(R, g.h)
    T, A = orc.fan_maps(g, c, tx, R, 0.05, K)
    maps = rt.BornMaps(g, R, torch.as_tensor(T, dtype=torch.float32, device="cuda"),
                       torch.as_tensor(A, dtype=torch.float32, device="cuda"))
    dc = P.SplitMix64(3).normal(g.nx * g.ny).reshape(g.ny, g.nx)
    d = rt.rtborn_apply(maps, [0.5, 1.0], torch.as_tensor(dc, dtype=torch.float32, device="cuda"), gemm="tf32x3")
    ref = orc.born_apply(g, R, T, A, np.array([0.5, 1.0]), dc)
    e = np.linalg.norm(d.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert np.isfinite(d.cpu().numpy()).all() and e <= 1e-4, e
