"""The sampling probabilities of the tracer's coin (Eq. path-solver-used-
dist-event with q(D) = 0: q(R) = wR / (wR + wT) from the coefficients of
Eqs. fresnel_vac, fresnel_slab, q_fresnel_slab) against the FP64 oracle at
the same FP32 cosines of incidence, through the tracer's own device code
(rm_debug_fresnel_probe).

The replay check adopts a GPU decision that differs from the oracle's when
the variate lies within a window of q(R): 1e-5 plus the change of q(R) when
the slab phase (2 pi d / lambda0) s moves by 2^-20 of itself.  The kernel's
own arithmetic must use at most a quarter of that window (the change under a
2^-22 relative phase change plus 2.5e-6); the rest covers the FP32 incidence
angle, whose relative phase error is at most |d cos| / (eps_r - 1)."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _q(orc, eps, sig, f, cos1, d):
    rp, rl, tp, tl = orc.fresnel(eps, sig, f, cos1, d)
    wR = abs(rp) ** 2 + abs(rl) ** 2
    wT = abs(tp) ** 2 + abs(tl) ** 2
    return wR / (wR + wT)


@pytest.mark.parametrize("cfg", [1, 2, 4, 5])
def test_coin_probabilities_vs_oracle(orc, api, cfg):
    from paper_2504_21719_b300 import _lib as L
    lib = L.load()
    sc, _, p = S.workload(cfg)
    rng = np.random.default_rng(cfg)
    cos1 = np.concatenate([np.linspace(0.0, 1.0, 2049), rng.uniform(0.0, 1.0, 2048),
                           [1e-6, 1e-3, 0.999999]]).astype(np.float32)
    cd = torch.tensor(cos1, device="cuda")
    wR = torch.empty_like(cd)
    wT = torch.empty_like(cd)
    worst = 0.0
    for m in sc.mats:
        mat = L.rm_material(float(m[0]), float(m[1]), float(m[2]))
        rc = lib.rm_debug_fresnel_probe(C.byref(mat), p.freq_hz, C.c_void_p(cd.data_ptr()), len(cos1),
                                        C.c_void_p(wR.data_ptr()), C.c_void_p(wT.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == L.RM_OK, lib.rm_last_error()
        torch.cuda.synchronize()
        r, t = wR.double().cpu().numpy(), wT.double().cpu().numpy()
        qg = r / (r + t)
        eps, sig, d = (float(np.float32(v)) for v in m)
        for i, c in enumerate(cos1.astype(np.float64)):
            q = _q(orc, eps, sig, p.freq_hz, c, d)
            allow = 2.5e-6 + 2.0 ** -22          # + the kernel's FP32 quotient wR / (wR + wT)
            win = 1e-5
            if d > 0:
                for fct in (1 - 2.0 ** -22, 1 + 2.0 ** -22):
                    allow = max(allow, 2.5e-6 + 2.0 ** -22 + abs(_q(orc, eps, sig, p.freq_hz, c, d * fct) - q))
                for fct in (1 - 2.0 ** -20, 1 + 2.0 ** -20):
                    win = max(win, 1e-5 + abs(_q(orc, eps, sig, p.freq_hz, c, d * fct) - q))
            dev = abs(qg[i] - q)
            assert dev <= allow, (m, c, qg[i], q, allow)
            worst = max(worst, dev / win)
    # the kernel's arithmetic uses at most a quarter of the replay's window
    assert worst <= 0.25, worst


def test_coin_record_changes_only_the_coin_bits(api):
    """RM_RECORD_COIN adds the coin's q(R) to the decision field and nothing
    else: same hits, cells, decisions and kill bits, q(R) in [0, 1], maps equal
    to the order of the atomic additions."""
    import copy
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 997
    gs = api.Scene.from_obj(sc)
    a = api.trace(gs, [tx], p, record=True)
    q = copy.copy(p)
    q.record_coin = True
    b = api.trace(gs, [tx], q, record=True)
    ra, rb = a["record"], b["record"]
    assert torch.equal(ra[:, :3], rb[:, :3])
    da, db = ra[:, 3], rb[:, 3]
    neg = da < 0
    assert torch.equal(da[neg], db[neg])
    assert torch.equal(da[~neg], db[~neg] & 255)
    coin = (db[~neg] >> 8).double() * 2.0 ** -22
    assert int((~neg).sum()) > 1000 and float(coin.min()) >= 0.0 and float(coin.max()) <= 1.0
    assert float((coin > 0).double().mean()) > 0.5
    ma, mb = a["maps"].double(), b["maps"].double()
    mask = ma > 1e-15
    assert torch.all((ma - mb).abs()[mask] <= 2e-5 * ma[mask])
    gs.free()
