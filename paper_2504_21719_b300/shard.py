"""Sharding of one radio map over several processes.

Rays are independent, so the lattice subset of every transmitter is split by
residue: rank r of W traces subset items i = r, r + W, r + 2W, ...  Each
rank's maps carry the full solid-angle weight 4 pi / N_S, so the maps of all
ranks add up to the map of the whole subset; one sum all-reduce of the maps
(the only collective) finishes the job.  The scene is replicated.

The adjoint shards the same way: the gradient of sum_i g_i C_i is linear in
the rays, so each rank differentiates its share with the same dL/dC (broadcast
from rank 0) and one sum all-reduce of the 2 nm + 3 ntx gradient values
finishes it.
"""
from __future__ import annotations

import copy


def partition_subset(begin: int, count: int, stride: int, rank: int, world: int):
    """(begin, count, stride) of rank's share of the items begin + i*stride, i < count."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    c = max(0, (count - rank + world - 1) // world)
    return begin + rank * stride, c, stride * world


def partition_tx(tx, rank: int, world: int):
    """A copy of transmitter `tx` restricted to rank's share of its rays.

    Works for any object with num_rays / ray_begin / ray_count / ray_stride
    attributes (ray_count < 0, None or UINT64_MAX = all)."""
    try:
        import ctypes
        t = type(tx).from_buffer_copy(tx) if isinstance(tx, ctypes.Structure) else copy.copy(tx)
        if isinstance(tx, ctypes.Structure) and hasattr(tx, "_keep"):
            t._keep = tx._keep  # antenna buffers referenced by pointer
    except Exception:
        t = copy.copy(tx)
    cnt = tx.ray_count
    if cnt is None or cnt < 0 or cnt >= (1 << 63):
        cnt = max(0, (tx.num_rays - tx.ray_begin + tx.ray_stride - 1) // tx.ray_stride)
    t.ray_begin, t.ray_count, t.ray_stride = partition_subset(tx.ray_begin, cnt, tx.ray_stride, rank, world)
    return t


def allreduce_maps(maps, group=None):
    """Sum the maps of all ranks in place (the only collective of a sharded trace)."""
    import torch.distributed as dist
    dist.all_reduce(maps, op=dist.ReduceOp.SUM, group=group)
    return maps


def sharded_trace(scene, txs, params, group=None, keep_hits=False):
    """Trace this rank's share of every transmitter and all-reduce the maps.  With
    keep_hits the result also holds this rank's recorded closest hits, for
    sharded_grad(..., hits=...) on the same rank."""
    import torch.distributed as dist

    from . import api
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    mine = [partition_tx(api.tx_from(t) if not hasattr(t, "_fields_") else t, rank, world) for t in txs]
    r = api.trace(scene, mine, params, keep_hits=keep_hits)
    allreduce_maps(r["maps"], group)
    return r


def allreduce_grads(grads, group=None):
    """Sum the gradient tensors (dict of d_eps, d_sigma, d_tx) of all ranks in place."""
    import torch
    import torch.distributed as dist
    flat = torch.cat([grads["d_eps"].reshape(-1), grads["d_sigma"].reshape(-1), grads["d_tx"].reshape(-1)])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    a, b = grads["d_eps"].numel(), grads["d_sigma"].numel()
    grads["d_eps"].copy_(flat[:a].view_as(grads["d_eps"]))
    grads["d_sigma"].copy_(flat[a:a + b].view_as(grads["d_sigma"]))
    grads["d_tx"].copy_(flat[a + b:].view_as(grads["d_tx"]))
    return grads


def sharded_grad(scene, txs, params, dLdC, group=None, src=0, hits=None):
    """Differentiate this rank's share of every transmitter with dL/dC
    broadcast from rank `src`, and all-reduce the gradients.  hits: this rank's
    sharded_trace(..., keep_hits=True)["hits"], replayed instead of traversing."""
    import torch.distributed as dist

    from . import api
    dist.broadcast(dLdC, src=src, group=group)
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    mine = [partition_tx(api.tx_from(t) if not hasattr(t, "_fields_") else t, rank, world) for t in txs]
    g = api.grad(scene, mine, params, dLdC, hits=hits)
    return allreduce_grads(g, group)
