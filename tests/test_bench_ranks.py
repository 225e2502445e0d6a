"""The benchmark's multi-rank bookkeeping on CPU (gloo, world size 2): every
rank's workload is a distinct 16-transmitter city workload, and the whole-job
figures take the slowest rank's time and the sum of every rank's segments and
copied bytes."""
import os
import socket

import numpy as np


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, counts = bench.over_ranks(dist, torch, 10.0 + 5.0 * rank, [100.0 * (rank + 1), 7.0, 2.0 ** 40 + rank], "cpu")
    if rank == 0:
        np.save(out, np.array([ms, *counts], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_over_ranks_max_time_and_summed_counts(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    out = str(tmp_path / "r.npy")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    got = np.load(out)
    assert got[0] == 15.0                                   # the slowest rank
    assert got[1] == 300.0 and got[2] == 14.0
    assert got[3] == 2.0 ** 41 + 1                          # byte counts stay exact in FP64


def test_rank_workloads_are_disjoint_and_extend_the_city():
    """Weak scaling: rank r of N traces transmitters 16 r .. 16 r + 15 of one
    seeded draw of 16 N; the first 16 are the one-GPU city workload's, and no
    two ranks share a transmitter position or random stream."""
    from synth import scenes as S
    sc, txs, _ = S.workload(5)
    for world in (1, 2, 4, 8):
        draw = S.city_transmitters(sc, 16 * world)
        ranks = [draw[16 * r:16 * (r + 1)] for r in range(world)]
        assert all(len(rk) == 16 for rk in ranks)
        assert [t.pos for t in ranks[0]] == [t.pos for t in txs]
        assert [t.seed for t in ranks[0]] == [t.seed for t in txs]
        assert len({t.pos for t in draw}) == 16 * world and len({t.seed for t in draw}) == 16 * world
