"""Multi-process path on CPU (gloo, world size 2): each rank's lattice share
of the rays, traced by the FP64 oracle, all-reduced, equals the whole map;
the same for the adjoint's gradient (dL/dC broadcast, gradients all-reduced)."""
import os
import socket

import numpy as np
import pytest

from synth import scenes as S


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup():
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride, tx.ray_begin = 2003, 11
    p.nx = p.ny = 128
    p.cell_size = 4.0
    return sc, tx, p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2504_21719_b300.shard import allreduce_maps, partition_tx
    sc, tx, p = _setup()
    mine = partition_tx(tx, rank, world)
    m = torch.from_numpy(oracle.radio_map(sc, mine, p)["map"])
    allreduce_maps(m)
    if rank == 0:
        np.save(out, m.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_partition_covers_every_item_once():
    from paper_2504_21719_b300.shard import partition_subset
    for count in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            items = []
            for r in range(world):
                b, c, s = partition_subset(5, count, 3, r, world)
                items += [b + i * s for i in range(c)]
            assert sorted(items) == [5 + 3 * i for i in range(count)]
    with pytest.raises(ValueError):
        partition_subset(0, 10, 1, 2, 2)


@pytest.mark.parametrize("world", [2])
def test_sharded_oracle_maps_sum_to_full_map(orc, tmp_path, world):
    import torch.multiprocessing as mp
    out = str(tmp_path / "m.npy")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    sc, tx, p = _setup()
    full = orc.radio_map(sc, tx, p)["map"]
    got = np.load(out)
    assert full.sum() > 0
    assert np.allclose(got, full, rtol=1e-12, atol=0)


def _grad_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2504_21719_b300.shard import allreduce_grads, partition_tx
    sc, tx, p = _setup()
    p.deposit = 1
    rng = np.random.default_rng(7)
    g = torch.from_numpy(rng.uniform(0.0, 1.0, (p.ny, p.nx)) if rank == 0 else np.zeros((p.ny, p.nx)))
    dist.broadcast(g, src=0)                      # dL/dC from rank 0
    mine = partition_tx(tx, rank, world)
    rec = oracle.radio_map(sc, mine, p, want_record=True)["record"]
    de, ds, dt = oracle.grad(sc, mine, p, rec, g.numpy())
    grads = {"d_eps": torch.from_numpy(de), "d_sigma": torch.from_numpy(ds), "d_tx": torch.from_numpy(dt).view(1, 3)}
    allreduce_grads(grads)
    if rank == 0:
        np.save(out, np.concatenate([grads["d_eps"].numpy(), grads["d_sigma"].numpy(), grads["d_tx"].numpy().ravel()]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_oracle_gradients_sum_to_full_gradient(orc, tmp_path):
    import torch.multiprocessing as mp
    world = 2
    out = str(tmp_path / "g.npy")
    mp.spawn(_grad_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    sc, tx, p = _setup()
    p.deposit = 1
    g = np.random.default_rng(7).uniform(0.0, 1.0, (p.ny, p.nx))
    rec = orc.radio_map(sc, tx, p, want_record=True)["record"]
    full = np.concatenate(orc.grad(sc, tx, p, rec, g))
    got = np.load(out)
    assert np.abs(full).max() > 0
    assert np.allclose(got, full, rtol=1e-10, atol=1e-12 * np.abs(full).max())
