"""Multi-rank path on CPU (gloo, world size 2): emitter sharding plus one
all-reduce of the adjoint reproduces the unsharded adjoint."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2511_18511_gb300 import shard  # noqa: E402


def test_shards_partition_all_pairs():
    from paper_2511_18511_gb300 import phantoms as P
    for n_tx, world in ((64, 2), (64, 3), (7, 4), (512, 8)):
        parts = [shard.shard_pairs(r, world, n_tx) for r in range(world)]
        allp = np.concatenate(parts)
        np.testing.assert_array_equal(allp, P.all_pairs(n_tx))
        idx = np.concatenate([shard.global_index(p, n_tx) for p in parts])
        np.testing.assert_array_equal(idx, np.arange(n_tx * (n_tx - 1)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2511_18511_gb300 import phantoms as P
    w = P.cfg_small(n_tx=16)
    pairs = shard.shard_pairs(rank, world, w.n_tx)
    r = oracle.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, pairs=pairs, nthreads=1)
    g_all = P.SplitMix64(3).normal(w.n_pairs)
    g = g_all[shard.global_index(pairs, w.n_tx)]
    gc = oracle.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"], g, pairs=pairs, nthreads=1)
    t = torch.from_numpy(gc.copy())
    shard.allreduce_sum(t)
    if rank == 0:
        np.save(os.path.join(out_dir, "sharded.npy"), t.numpy())
    dist.destroy_process_group()


def test_sharded_adjoint_equals_unsharded(tmp_path, orc):
    from paper_2511_18511_gb300 import phantoms as P
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    sharded = np.load(tmp_path / "sharded.npy")
    w = P.cfg_small(n_tx=16)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds)
    g_all = P.SplitMix64(3).normal(w.n_pairs)
    full = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"], g_all)
    assert np.abs(sharded - full).max() <= 1e-13 * np.abs(full).max()


def test_frequency_blocks_partition():
    for n_freq, world in ((8, 2), (8, 3), (3, 4), (1, 2), (16, 8)):
        parts = [shard.frequencies_of(r, world, n_freq) for r in range(world)]
        np.testing.assert_array_equal(np.concatenate(parts), np.arange(n_freq))


def _born_case():
    from paper_2511_18511_gb300 import phantoms as P
    from tests.test_oracle_born_pins import _synthetic_maps
    g = P.Grid(24, 24, 0.5)
    R = 5.5
    tx = P.ring(6, R)
    T, A = _synthetic_maps(g, tx, 3)
    f = P.born_frequencies(5)
    rng = P.SplitMix64(17)
    dc = rng.normal(g.nx * g.ny).reshape(g.ny, g.nx)
    n = len(f) * len(tx) ** 2
    d = (rng.normal(n) + 1j * rng.normal(n)).reshape(len(f), len(tx), len(tx))
    return g, R, T, A, f, dc, d


def _born_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    g, R, T, A, f, dc, d = _born_case()
    mine = shard.frequencies_of(rank, world, len(f))
    d_loc = oracle.born_apply(g, R, T, A, f[mine], dc, nthreads=1)
    d_all = shard.allgather_frequencies(torch.from_numpy(d_loc.copy()), len(f))
    adj = torch.from_numpy(oracle.born_adjoint(g, R, T, A, f[mine], d[mine], nthreads=1).copy())
    shard.allreduce_sum(adj)
    if rank == 0:
        np.save(os.path.join(out_dir, "born_apply.npy"), d_all.numpy())
        np.save(os.path.join(out_dir, "born_adjoint.npy"), adj.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_born_frequency_sharding_equals_unsharded(tmp_path, orc, world):
    """Ray-Born over ranks: each rank applies the Born map for its block of the
    5 frequencies (3 ranks: blocks of 1, 2, 2), one all-gather assembles the
    data, and the adjoint of each rank's block summed by one all-reduce equals
    the unsharded adjoint."""
    mp.start_processes(_born_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    g, R, T, A, f, dc, d = _born_case()
    full = orc.born_apply(g, R, T, A, f, dc)
    got = np.load(tmp_path / "born_apply.npy")
    assert got.shape == full.shape
    np.testing.assert_array_equal(got, full)
    adj = orc.born_adjoint(g, R, T, A, f, d)
    got_adj = np.load(tmp_path / "born_adjoint.npy")
    assert np.abs(got_adj - adj).max() <= 1e-13 * np.abs(adj).max()


def test_longest_first_shards_partition_all_pairs():
    """The longest-first order of a shard is a permutation of its pairs, with
    ring distances non-increasing."""
    for n_tx, world in ((64, 2), (64, 3), (512, 8)):
        for r in range(world):
            a = shard.shard_pairs(r, world, n_tx)
            b = shard.shard_pairs(r, world, n_tx, longest_first=True)
            assert {tuple(p) for p in a} == {tuple(p) for p in b} and len(a) == len(b)
            off = (b[:, 1] - b[:, 0]) % n_tx
            far = np.minimum(off, n_tx - off)
            assert (np.diff(far) <= 0).all()


def _step_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2511_18511_gb300 import phantoms as P
    w = P.cfg_small(n_tx=16)

    def link(pairs, c):
        r = oracle.link(w.grid, c, w.tx, w.ring_radius, w.ds, pairs=pairs, nthreads=1, fan_rays=64)
        return r["theta"], r["tof"]

    def adjoint(pairs, c, theta, tof, tof_meas):
        return torch.from_numpy(oracle.adjoint(w.grid, c, w.tx, w.ring_radius, w.ds, theta, tof - tof_meas,
                                               pairs=pairs, nthreads=1).copy())

    def link_adjoint(pairs, c, tof_meas):
        theta, tof = link(pairs, c)
        return theta, tof, adjoint(pairs, c, theta, tof, tof_meas)

    step = shard.ShardedToF(rank, world, w.n_tx, link, adjoint)
    _, t_meas = link(step.pairs, w.c * 1.005)
    g, _, _ = step.step(w.c, t_meas)
    fused = shard.ShardedToF(rank, world, w.n_tx, link_adjoint=link_adjoint)
    g2, _, _ = fused.step(w.c, t_meas)
    if rank == 0:
        np.save(os.path.join(out_dir, "step.npy"), g.numpy())
        np.save(os.path.join(out_dir, "step_fused.npy"), g2.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_tof_step_equals_unsharded(tmp_path, orc, world):
    """The step the bench runs on N GPUs (ShardedToF: link and misfit adjoint
    of each rank's longest-first emitter block, then one all-reduce), run with
    the oracle's operators on gloo ranks: the summed gradient equals the
    unsharded step's."""
    from paper_2511_18511_gb300 import phantoms as P
    mp.start_processes(_step_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "step.npy")
    np.testing.assert_array_equal(np.load(tmp_path / "step_fused.npy"), got)
    w = P.cfg_small(n_tx=16)
    meas = orc.link(w.grid, w.c * 1.005, w.tx, w.ring_radius, w.ds, fan_rays=64)
    r = orc.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, fan_rays=64)
    full = orc.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"], r["tof"] - meas["tof"])
    assert np.abs(got - full).max() <= 1e-13 * np.abs(full).max()


def _failing_rank_worker(rank, world, port, out_dir):
    """Rank 1 fails in its link before the step's all-reduce; rank 0 must see an
    error from its all-reduce within the process group's timeout, not hang."""
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    n_tx = 8

    def link(pairs, c):
        if rank == 1:
            raise RuntimeError("link failed on rank 1")
        return np.zeros(len(pairs)), np.zeros(len(pairs))

    def adjoint(pairs, c, theta, tof, tof_meas):
        return torch.ones(16, dtype=torch.float64)

    step = shard.ShardedToF(rank, world, n_tx, link=link, adjoint=adjoint)
    t0 = time.time()
    try:
        step.step(None, np.zeros(len(step.pairs)))
        outcome = "completed"
    except Exception as exc:   # the failing rank's own error, or the survivor's collective error
        outcome = type(exc).__name__
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{outcome} {time.time() - t0:.2f}\n")
    if rank == 1:
        os._exit(0)            # leave without the collective, as a failed rank would


def test_sharded_step_reports_a_failed_rank(tmp_path):
    """Failure detection on the host: a rank that raises inside the step leaves
    before the all-reduce; the other rank's all-reduce ends with an error within
    the process group's timeout instead of hanging."""
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=60)
    alive = [p.is_alive() for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert not any(alive), alive
    r0 = (tmp_path / "rank0.txt").read_text().split()
    r1 = (tmp_path / "rank1.txt").read_text().split()
    print(f"rank 0: {r0}, rank 1: {r1}")
    assert r1[0] == "RuntimeError"
    assert r0[0] != "completed" and float(r0[1]) < 30.0
