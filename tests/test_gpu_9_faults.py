"""Injected host-side failures on a real device: each returns its status, no
kernel faults, and the next call on the same context is correct."""
import pytest
import torch

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _small():
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 101
    return sc, tx, p


def test_injected_launch_and_overflow_keep_the_context(api):
    from paper_2504_21719_b300 import _lib as L
    sc, tx, p = _small()
    gs = api.Scene.from_obj(sc)
    ref = api.trace(gs, [tx], p)["maps"].clone()
    lib = L.load()
    assert lib.rm_debug_inject(L.RM_FAULT_LAUNCH, 1) == L.RM_OK
    with pytest.raises(api.RmError, match="injected launch failure") as e:
        api.trace(gs, [tx], p)
    assert e.value.status == L.RM_ECUDA
    assert torch.equal(api.trace(gs, [tx], p)["maps"], ref)
    # an overflow report: the maps are written, the status says rays may be missing
    assert lib.rm_debug_inject(L.RM_FAULT_OVERFLOW, 1) == L.RM_OK
    out = torch.zeros_like(ref)
    with pytest.raises(api.RmError) as e:
        api.trace(gs, [tx], p, out=out)
    assert e.value.status == L.RM_EOVERFLOW
    assert torch.allclose(out, ref, rtol=2e-5, atol=0)
    # the adjoint reports the same way
    assert lib.rm_debug_inject(L.RM_FAULT_LAUNCH, 1) == L.RM_OK
    with pytest.raises(api.RmError, match="injected"):
        api.grad(gs, [tx], p, torch.ones_like(ref))
    g = api.grad(gs, [tx], p, torch.ones_like(ref))
    assert torch.isfinite(g["d_eps"]).all()
    assert torch.allclose(api.trace(gs, [tx], p)["maps"], ref, rtol=2e-5, atol=0)
    gs.free()


def test_injected_allocation_failure_then_upload(api):
    from paper_2504_21719_b300 import _lib as L
    sc, tx, p = _small()
    assert L.load().rm_debug_inject(L.RM_FAULT_ALLOC, 1) == L.RM_OK
    with pytest.raises(api.RmError) as e:
        api.Scene.from_obj(sc)
    assert e.value.status == L.RM_ENOMEM
    gs = api.Scene.from_obj(sc)
    assert float(api.trace(gs, [tx], p)["maps"].sum()) > 0.0
    gs.free()
