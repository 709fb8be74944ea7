"""Batched persistent launch (rt_batch_run): uneven instances in one launch,
against the single-problem calls and the oracle, replayed from a CUDA graph,
and the autotuner."""
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


@pytest.fixture(scope="module")
def P():
    from paper_2511_18511_gb300 import phantoms
    return phantoms


def _np(t):
    return t.detach().cpu().numpy()


def _small_batch(P, rt):
    """Four uneven instances (grids 96^2..160^2 at 0.5 mm, rings 12..32) with
    measured times from a 1%-faster medium, and one without an adjoint."""
    specs = [(96, 12, 11), (160, 32, 12), (128, 24, 13), (112, 16, 14)]
    out = []
    for n, nt, seed in specs:
        g = P.Grid(n, n, 0.5)
        R = 0.45 * n * 0.5
        c = P.gaussian_inclusions(g, seed, centre_radius=0.6 * R, sigma_lo=2.0, sigma_hi=5.0)
        prob = rt.Problem.create(g, c, P.ring(nt, R), R)
        ref = rt.rt_link(prob, 0.05, precision="fp64", c=prob.c * 1.01)["tof"].clone()
        out.append((g, c, P.ring(nt, R), R, prob, ref))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_batch_equals_single_calls_and_oracle(rt, P, orc, prec):
    ds, tol = 0.05, 1e-4
    items = _small_batch(P, rt)
    insts = [rt.BatchInstance.create(it[4], tof_ref=(it[5] if k != 3 else None)) for k, it in enumerate(items)]
    rt.rt_batch_run(insts, ds, tol, precision=prec)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == sum(it[4].n_pairs for it in items)
    for k, (g, c, tx, R, prob, ref) in enumerate(items):
        b = insts[k]
        single = rt.rt_link(prob, ds, tol=tol, precision=prec)
        np.testing.assert_allclose(_np(b.tof), _np(single["tof"]), rtol=1e-12 if prec == "fp64" else 1e-9)
        np.testing.assert_array_equal(_np(b.iters), _np(single["iters"]))
        o = orc.link(g, c, tx, R, ds, tol=tol, fan_rays=rt.DEFAULT_FAN)
        rel = np.abs(_np(b.tof) / o["tof"] - 1).max()
        assert rel <= (1e-12 if prec == "fp64" else 2e-6), rel
        if b.tof_ref is None:
            continue
        g_single = rt.rt_tof_adjoint(prob, single["theta"], single["tof"], ds, tof_ref=ref, precision=prec)
        a, s_ = _np(b.g_c), _np(g_single)
        assert np.linalg.norm(a - s_) <= 1e-12 * np.linalg.norm(s_) if prec == "fp64" else \
            np.linalg.norm(a - s_) <= 1e-6 * np.linalg.norm(s_)
        want = orc.adjoint(g, c, tx, R, ds, o["theta"], o["tof"] - _np(ref))
        e = np.linalg.norm(a - want) / np.linalg.norm(want)
        print(f"[{prec}] instance {k}: ToF vs oracle {rel:.2e}, adjoint vs oracle {e:.2e}")
        assert e <= 1e-5


def test_batch_with_coarse_fan_equals_single_calls_and_oracle(rt, P, orc):
    """The bench's batch setting, fans traced at h/2 (FP32-compensated): the
    batch links as the single calls with the same fan step, travel times within
    the linking bar of the oracle's with the same fan step; a sub-fan option is
    refused (the batch links in one launch)."""
    ds, tol = 0.05, 1e-4
    items = _small_batch(P, rt)
    fds = 0.5 * items[0][0].h
    insts = [rt.BatchInstance.create(it[4], tof_ref=it[5]) for it in items]
    rt.rt_batch_run(insts, ds, tol, fan_ds=fds)
    ok, counts = rt.rt_status_counts()
    assert ok and counts[0] == sum(it[4].n_pairs for it in items)
    for k, (g, c, tx, R, prob, ref) in enumerate(items):
        b = insts[k]
        single = rt.rt_link(prob, ds, tol=tol, fan_ds=fds)
        np.testing.assert_allclose(_np(b.tof), _np(single["tof"]), rtol=1e-9)
        np.testing.assert_array_equal(_np(b.iters), _np(single["iters"]))
        o = orc.link(g, c, tx, R, ds, tol=tol, fan_rays=rt.DEFAULT_FAN, fan_ds=fds)
        rel = np.abs(_np(b.tof) / o["tof"] - 1).max()
        print(f"[fan at h/2] instance {k}: ToF vs oracle {rel:.2e}, traces/pair {_np(b.iters).mean():.3f} "
              f"(oracle {o['iters'].mean():.3f})")
        assert rel <= 2e-6
    o = rt._opts(ds, tol, subfan_rays=8)
    with pytest.raises(rt._L.RtError):
        _batch_with_opts(rt, insts, o)


def _batch_with_opts(rt, insts, o):
    ctx = rt.default_context(insts[0].prob.c.device.index)
    arr = (rt._L.RtInstance * len(insts))(*[b.struct() for b in insts])
    rt._L.check(ctx.h, ctx.lib.rt_batch_run(ctx.h, len(insts), arr, C.byref(o), None))


def test_batch_graph_replay(rt, P):
    ds = 0.05
    items = _small_batch(P, rt)
    insts = [rt.BatchInstance.create(it[4], tof_ref=it[5]) for it in items]
    rt.rt_batch_run(insts, ds)                    # sizes the workspace outside capture
    torch.cuda.synchronize()
    eager = [(_np(b.tof).copy(), _np(b.g_c).copy()) for b in insts]
    for b in insts:
        b.theta.fill_(float("nan"))
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            rt.rt_batch_run(insts, ds, reset_angles=False, stream=s)
    for _ in range(2):
        for b in insts:
            b.theta.fill_(float("nan"))
            b.tof.zero_()
            b.g_c.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for b, (T0, g0) in zip(insts, eager):
            np.testing.assert_allclose(_np(b.tof), T0, rtol=1e-12)
            np.testing.assert_allclose(_np(b.g_c), g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max())


def test_autotuner_and_bad_options(rt, P, tmp_path, monkeypatch):
    from paper_2511_18511_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    items = _small_batch(P, rt)
    insts = [rt.BatchInstance.create(it[4], tof_ref=it[5]) for it in items]
    best, times = autotune.tune_batch(insts, 0.05, reps=1)
    assert best in autotune.CANDIDATES and len(times) == len(autotune.CANDIDATES)
    best2, _ = autotune.tune_batch(insts, 0.05)          # from the cache
    assert best2 == best
    with pytest.raises(rt._L.RtError):
        rt.rt_batch_run(insts, 0.05, block_threads=96)
    with pytest.raises(rt._L.RtError):
        rt.rt_batch_run(insts, 0.05, precision="fp64", block_threads=256)
    with pytest.raises(rt._L.RtError):
        rt.rt_batch_run(insts, 0.05, block_threads=128, blocks_per_sm=7)
    L = rt._L.load()
    ctx = rt.default_context()
    o = rt._opts(0.05)
    arr = (rt._L.RtInstance * 65)()
    assert L.rt_batch_run(ctx.h, 65, arr, C.byref(o), None) == rt._L.RT_EINVAL
