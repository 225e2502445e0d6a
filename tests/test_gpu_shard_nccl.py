"""The sharded map and gradient (one sum all-reduce each) through the CUDA
path and NCCL at world size 1: the partition of one rank is the whole lattice
subset, so the sharded results equal api.trace / api.grad.  (Each box has one
GPU; the world-size-2 collective logic runs on CPU with gloo.)"""
import socket

import pytest
import torch

from synth import scenes as S
from gpu_helpers import FLOOR

pytestmark = pytest.mark.gpu


@pytest.fixture
def nccl_group():
    import torch.distributed as dist
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    yield dist
    dist.destroy_process_group()


def test_sharded_trace_and_grad_world_size_1(api, nccl_group):
    from paper_2504_21719_b300.shard import sharded_grad, sharded_trace
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = 5
    gs = api.Scene.from_obj(sc)
    ref = api.trace(gs, [tx], p)
    sh = sharded_trace(gs, [tx], p)
    torch.cuda.synchronize()
    a, b = sh["maps"].double(), ref["maps"].double()
    mask = b > FLOOR
    assert int(mask.sum()) > 1000
    assert torch.all((a - b).abs()[mask] <= 2e-5 * b[mask])
    assert sh["stats"]["segments"] == ref["stats"]["segments"]
    g = torch.rand_like(ref["maps"]) * 1e-3
    gr = api.grad(gs, [tx], p, g)
    gsh = sharded_grad(gs, [tx], p, g.clone())
    for key in ("d_eps", "d_sigma", "d_tx"):
        x, y = gsh[key].double(), gr[key].double()
        scale = y.abs().max().item()
        assert scale > 0
        assert torch.all((x - y).abs() <= 1e-4 * scale), (key, x, y)
    # the same with the forward's hits recorded and replayed by the adjoint
    shh = sharded_trace(gs, [tx], p, keep_hits=True)
    assert torch.all((shh["maps"].double() - b).abs()[mask] <= 2e-5 * b[mask])
    gsh2 = sharded_grad(gs, [tx], p, g.clone(), hits=shh["hits"])
    for key in ("d_eps", "d_sigma", "d_tx"):
        x, y = gsh2[key].double(), gr[key].double()
        scale = y.abs().max().item()
        assert torch.all((x - y).abs() <= 1e-4 * scale), (key, x, y)
    gs.free()
