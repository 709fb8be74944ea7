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
