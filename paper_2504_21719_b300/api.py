"""PyTorch-facing helpers over the C ABI.

PyTorch provides device memory and the current stream; every computation of
the radio-map path happens inside librmsbr.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


class RmError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = L.load().rm_last_error().decode()
        super().__init__(f"{where}: {L.STATUS_NAMES[status]}: {msg}")
        self.status = status


def _check(status: int, where: str):
    if status != L.RM_OK:
        raise RmError(status, where)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def materials(mats, scat=None) -> C.Array:
    """Array of rm_material from an [nm, 3] (eps_r, sigma, thickness) table and
    optional diffuse parameters [nm, 6] = (S, K_x, pattern, alpha_R, alpha_I, Lambda)."""
    m = np.asarray(mats, np.float64).reshape(-1, 3)
    sc = None if scat is None else np.asarray(scat, np.float64).reshape(-1, 6)
    if sc is not None and len(sc) != len(m):
        raise ValueError("scat must have one row per material")
    arr = (L.rm_material * len(m))()
    for i, (e, s, d) in enumerate(m):
        x = L.rm_material(float(e), float(s), float(d))
        if sc is not None:
            x.scattering, x.xpd_k = float(sc[i, 0]), float(sc[i, 1])
            x.pattern, x.alpha_r, x.alpha_i = int(sc[i, 2]), int(sc[i, 3]), int(sc[i, 4])
            x.lobe_lambda = float(sc[i, 5])
        arr[i] = x
    return arr


def tx_struct(pos, num_rays, yaw=0.0, pitch=0.0, roll=0.0, pol=0, pattern=0, ray_begin=0, ray_count=None,
              ray_stride=1, seed=0, ant_pos=None, precoding=None) -> L.rm_tx:
    t = L.rm_tx()
    if ant_pos is not None and len(ant_pos):
        a = np.ascontiguousarray(np.asarray(ant_pos, np.float64).reshape(-1, 3))
        w = np.asarray(precoding, np.complex128).reshape(-1)
        pc = np.ascontiguousarray(np.stack([w.real, w.imag], 1), np.float64)
        t._keep = (a, pc)  # the buffers live as long as the struct
        t.n_ant = len(a)
        t.ant_pos_host = a.ctypes.data
        t.precoding_host = pc.ctypes.data
    for i in range(3):
        t.pos[i] = float(pos[i])
    t.yaw, t.pitch, t.roll = float(yaw), float(pitch), float(roll)
    t.pol, t.pattern = int(pol), int(pattern)
    t.num_rays, t.ray_begin, t.ray_stride = int(num_rays), int(ray_begin), int(ray_stride)
    t.ray_count = L.UINT64_MAX if ray_count is None or ray_count < 0 else int(ray_count)
    t.seed = int(seed)
    return t


def tx_from(obj) -> L.rm_tx:
    """rm_tx from any object with the rm_tx field names as attributes."""
    return tx_struct(obj.pos, obj.num_rays, obj.yaw, obj.pitch, obj.roll, obj.pol, obj.pattern, obj.ray_begin,
                     obj.ray_count, obj.ray_stride, obj.seed, getattr(obj, "ant_pos", None),
                     getattr(obj, "precoding", None))


def params_struct(freq_hz, max_depth, map_origin=(0.0, 0.0, 1.5), cell_size=1.0, nx=100, ny=100,
                  reflect=True, refract=True, los=True, stats=False, deposit=0, block_size=0,
                  blocks_per_sm=0, queue_chunk=0, rr_depth=0, rr_max_prob=0.0,
                  gain_threshold=0.0, diffuse=False, refill_min=0, record_coin=False) -> L.rm_trace_params:
    p = L.rm_trace_params()
    p.freq_hz = float(freq_hz)
    p.max_depth = int(max_depth)
    p.flags = ((L.RM_REFLECT if reflect else 0) | (L.RM_REFRACT if refract else 0) |
               (L.RM_LOS if los else 0) | (L.RM_STATS if stats else 0) | (L.RM_DIFFUSE if diffuse else 0) |
               (L.RM_RECORD_COIN if record_coin else 0))
    for i in range(3):
        p.map_origin[i] = float(map_origin[i])
    p.cell_size = float(cell_size)
    p.nx, p.ny, p.deposit = int(nx), int(ny), int(deposit)
    p.block_size, p.blocks_per_sm, p.queue_chunk = int(block_size), int(blocks_per_sm), int(queue_chunk)
    p.rr_depth, p.rr_max_prob, p.gain_threshold = int(rr_depth), float(rr_max_prob), float(gain_threshold)
    p.refill_min = int(refill_min)
    return p


def params_from(obj, stats=False, block_size=0, blocks_per_sm=0, queue_chunk=0, refill_min=0) -> L.rm_trace_params:
    return params_struct(obj.freq_hz, obj.max_depth, obj.map_origin, obj.cell_size, obj.nx, obj.ny, obj.reflect,
                         obj.refract, obj.los, stats, obj.deposit, block_size, blocks_per_sm, queue_chunk,
                         getattr(obj, "rr_depth", 0), getattr(obj, "rr_max_prob", 0.0),
                         getattr(obj, "gain_threshold", 0.0), getattr(obj, "diffuse", False), refill_min,
                         getattr(obj, "record_coin", False))


def _tx_array(txs):
    txs = [t if isinstance(t, L.rm_tx) else tx_from(t) for t in txs]
    arr = (L.rm_tx * len(txs))(*txs)
    # the copies in arr point at the antenna buffers that the structs keep alive
    arr._keep = [getattr(t, "_keep", None) for t in txs]
    return arr, len(txs)


def tx_count(t: L.rm_tx) -> int:
    if t.ray_count != L.UINT64_MAX:
        return int(t.ray_count)
    if t.ray_begin >= t.num_rays:
        return 0
    return (t.num_rays - t.ray_begin + t.ray_stride - 1) // t.ray_stride


class Scene:
    """A triangle mesh with per-triangle materials, uploaded and with its BVH built
    (``builder``: "auto", "lbvh" or "sah"; see rm_bvh_build_ex)."""

    BUILDERS = {"auto": 0, "lbvh": 1, "sah": 2}

    def __init__(self, verts, tris, tri_mat, mats, device="cuda", stream=None, build=True, scat=None,
                 builder="auto"):
        lib = L.load()
        dev = torch.device(device)

        def dev_tensor(a, dt_np, dt_t):
            if isinstance(a, torch.Tensor):
                return a.to(device=dev, dtype=dt_t, non_blocking=True).contiguous()
            return torch.as_tensor(np.ascontiguousarray(a, dt_np)).to(dev)

        self.nm = int(np.asarray(mats).reshape(-1, 3).shape[0])
        self._scat = None if scat is None else np.asarray(scat, np.float64).reshape(-1, 6)
        self._mats = materials(mats, self._scat)
        h = C.c_void_p()
        on_host = all(not (isinstance(a, torch.Tensor) and a.is_cuda) for a in (verts, tris, tri_mat))
        if on_host and dev.type == "cuda":
            # host arrays: checked on the host, one pinned asynchronous copy, no device round trip
            def host_array(a, dt_np):
                if isinstance(a, torch.Tensor):
                    a = a.numpy()
                return np.ascontiguousarray(a, dt_np)

            v = host_array(verts, np.float32).reshape(-1, 3)
            t = host_array(tris, np.int32).reshape(-1, 3)
            m = host_array(tri_mat, np.int32).reshape(-1)
            self.nt = int(t.shape[0])
            _check(lib.rm_scene_upload_host(v.ctypes.data, v.shape[0], t.ctypes.data, self.nt, m.ctypes.data,
                                            self._mats, self.nm, _stream(stream), C.byref(h)),
                   "rm_scene_upload_host")
        else:
            v = dev_tensor(verts, np.float32, torch.float32)
            t = dev_tensor(tris, np.int32, torch.int32)
            m = dev_tensor(tri_mat, np.int32, torch.int32)
            self.nt = int(t.shape[0])
            _check(lib.rm_scene_upload(_ptr(v), v.shape[0], _ptr(t), self.nt, _ptr(m), self._mats, self.nm,
                                       _stream(stream), C.byref(h)), "rm_scene_upload")
        self.handle = h
        if build:
            self.build_bvh(stream, builder)

    @classmethod
    def from_obj(cls, sc, **kw):
        return cls(sc.verts, sc.tris, sc.tri_mat, sc.mats, scat=getattr(sc, "scat", None), **kw)

    def build_bvh(self, stream=None, builder="auto"):
        _check(L.load().rm_bvh_build_ex(self.handle, self.BUILDERS[builder], _stream(stream)), "rm_bvh_build_ex")

    def set_materials(self, mats, sampling=None, scat=None):
        """Replace the materials; the diffuse parameters stay unless `scat` is given."""
        if scat is not None:
            self._scat = np.asarray(scat, np.float64).reshape(-1, 6)
        self._mats = materials(mats, self._scat)
        sm = None if sampling is None else materials(sampling)
        self._smats = sm
        _check(L.load().rm_scene_set_materials(self.handle, self._mats, self.nm, sm), "rm_scene_set_materials")

    def info(self):
        nt, nn, nm, built = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        _check(L.load().rm_scene_info(self.handle, C.byref(nt), C.byref(nn), C.byref(nm), C.byref(built)),
               "rm_scene_info")
        return {"nt": nt.value, "nodes": nn.value, "nm": nm.value, "built": bool(built.value),
                "builder": {0: None, 1: "lbvh", 2: "sah"}[built.value]}

    def export_bvh(self):
        n = self.nt
        nn = self.info()["nodes"]
        keys = np.zeros(max(n, 1), np.uint64)
        order = np.zeros(max(n, 1), np.int32)
        child = np.zeros((max(nn, 1), 2), np.int32)
        box = np.zeros((max(nn, 1), 2, 6), np.float32)
        _check(L.load().rm_bvh_export(self.handle, keys.ctypes.data_as(C.c_void_p), order.ctypes.data_as(C.c_void_p),
                                      child.ctypes.data_as(C.c_void_p), box.ctypes.data_as(C.c_void_p)),
               "rm_bvh_export")
        nlarge = int((keys[:n] == np.uint64(2 ** 64 - 1)).sum())
        return {"keys": keys[:n], "order": order[:n], "nlarge": nlarge, "child": child[:nn],
                "child_aabb": box[:nn]}

    def wedges(self):
        """ctypes array of rm_wedge: the scene's wedges ordered by (tri0, trin)."""
        n = C.c_int64()
        _check(L.load().rm_scene_wedges(self.handle, None, 0, C.byref(n)), "rm_scene_wedges")
        arr = (L.rm_wedge * max(n.value, 1))()
        _check(L.load().rm_scene_wedges(self.handle, arr, n.value, C.byref(n)), "rm_scene_wedges")
        self._wedges = arr
        self._nw = n.value
        return arr, n.value

    def free(self):
        if getattr(self, "handle", None):
            L.load().rm_scene_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def trace(scene: Scene, txs, params, record=False, stream=None, out=None, keep_hits=False, hits_out=None):
    """Radio maps [ntx, ny, nx] (float32, cuda) and the counters; optionally the per-segment
    record, or (keep_hits) every segment's closest-hit leaf slot for grad(..., hits=...),
    written into hits_out (int32, cuda) when it is given."""
    lib = L.load()
    arr, ntx = _tx_array(txs)
    p = params if isinstance(params, L.rm_trace_params) else params_from(params)
    maps = out if out is not None else torch.empty((ntx, p.ny, p.nx), dtype=torch.float32, device="cuda")
    if keep_hits:
        if record:
            raise ValueError("keep_hits and record are separate calls")
        nh = sum(tx_count(arr[i]) for i in range(ntx)) * (p.max_depth + 1)
        hits = hits_out if hits_out is not None else torch.empty(max(nh, 1), dtype=torch.int32, device="cuda")
        st = L.rm_stats()
        if hits.dtype != torch.int32 or not hits.is_cuda or not hits.is_contiguous():
            raise ValueError("hits_out must be a contiguous int32 cuda tensor")
        _check(lib.rm_radio_map_trace_hits(scene.handle, arr, ntx, C.byref(p), _ptr(maps), _ptr(hits), hits.numel(),
                                           C.byref(st), _stream(stream)), "rm_radio_map_trace_hits")
        return {"maps": maps, "stats": st.as_dict(), "hits": hits}
    rec = None
    if record:
        nrec = sum(tx_count(arr[i]) for i in range(ntx)) * (p.max_depth + 1)
        rec = torch.empty((max(nrec, 1), 4), dtype=torch.int32, device="cuda")
    st = L.rm_stats()
    _check(lib.rm_radio_map_trace(scene.handle, arr, ntx, C.byref(p), _ptr(maps), C.byref(st), _ptr(rec),
                                  _stream(stream)), "rm_radio_map_trace")
    res = {"maps": maps, "stats": st.as_dict()}
    if record:
        res["record"] = rec
    return res


def diffraction_map_mesh(scene: Scene, surface: Scene, txs, params, samples_per_wedge: int, wedges=None,
                         record=False, stream=None, out=None):
    """First-order diffraction maps [ntx, surface triangles] (float32, cuda) on a mesh
    measurement surface; add them to trace_mesh()'s maps for the full map."""
    lib = L.load()
    arr, ntx = _tx_array(txs)
    p = params if isinstance(params, L.rm_trace_params) else params_from(params)
    w, nw = wedges if wedges is not None else scene.wedges()
    maps = out if out is not None else torch.empty((ntx, surface.nt), dtype=torch.float32, device="cuda")
    rec = None
    if record:
        rec = torch.empty((max(ntx * nw * samples_per_wedge, 1), 4), dtype=torch.int32, device="cuda")
    st = L.rm_stats()
    _check(lib.rm_diffraction_map_mesh(scene.handle, surface.handle, w, nw, arr, ntx, C.byref(p),
                                       int(samples_per_wedge), _ptr(maps), C.byref(st), _ptr(rec), _stream(stream)),
           "rm_diffraction_map_mesh")
    res = {"maps": maps, "stats": st.as_dict(), "wedges": nw}
    if record:
        res["record"] = rec
    return res


def trace_mesh(scene: Scene, surface: Scene, txs, params, record=False, stream=None, out=None, keep_hits=False):
    """Radio maps on a mesh measurement surface: [ntx, surface triangles] (float32, cuda),
    one cell per triangle of `surface` (a Scene whose materials are unused); the counters;
    optionally the per-segment record, or (keep_hits) every segment's closest-hit leaf slot
    in the scene for grad_mesh(..., hits=...)."""
    lib = L.load()
    arr, ntx = _tx_array(txs)
    p = params if isinstance(params, L.rm_trace_params) else params_from(params)
    maps = out if out is not None else torch.empty((ntx, surface.nt), dtype=torch.float32, device="cuda")
    if keep_hits:
        if record:
            raise ValueError("keep_hits and record are separate calls")
        nh = sum(tx_count(arr[i]) for i in range(ntx)) * (p.max_depth + 1)
        hits = torch.empty(max(nh, 1), dtype=torch.int32, device="cuda")
        st = L.rm_stats()
        _check(lib.rm_radio_map_trace_mesh_hits(scene.handle, surface.handle, arr, ntx, C.byref(p), _ptr(maps),
                                                _ptr(hits), hits.numel(), C.byref(st), _stream(stream)),
               "rm_radio_map_trace_mesh_hits")
        return {"maps": maps, "stats": st.as_dict(), "hits": hits}
    rec = None
    if record:
        nrec = sum(tx_count(arr[i]) for i in range(ntx)) * (p.max_depth + 1)
        rec = torch.empty((max(nrec, 1), 4), dtype=torch.int32, device="cuda")
    st = L.rm_stats()
    _check(lib.rm_radio_map_trace_mesh(scene.handle, surface.handle, arr, ntx, C.byref(p), _ptr(maps), C.byref(st),
                                       _ptr(rec), _stream(stream)), "rm_radio_map_trace_mesh")
    res = {"maps": maps, "stats": st.as_dict()}
    if record:
        res["record"] = rec
    return res


def grad_mesh(scene: Scene, surface: Scene, txs, params, dLdC: torch.Tensor, sampling=None, record=False,
              stream=None, hits=None):
    """(d_eps [nm], d_sigma [nm], d_txpos [ntx, 3] = 0) of sum(dLdC * maps) for maps on a mesh
    measurement surface (dLdC [ntx, surface triangles]); choices frozen, q detached.
    hits: trace_mesh(..., keep_hits=True)["hits"] of the same arguments, replayed instead of
    traversing the scene's BVH."""
    lib = L.load()
    arr, ntx = _tx_array(txs)
    p = params if isinstance(params, L.rm_trace_params) else params_from(params)
    d_eps = torch.zeros(scene.nm, dtype=torch.float32, device="cuda")
    d_sig = torch.zeros(scene.nm, dtype=torch.float32, device="cuda")
    d_tx = torch.zeros((ntx, 3), dtype=torch.float32, device="cuda")
    sm = None if sampling is None else materials(sampling)
    rec = None
    if record:
        nrec = sum(tx_count(arr[i]) for i in range(ntx)) * (p.max_depth + 1)
        rec = torch.empty((max(nrec, 1), 4), dtype=torch.int32, device="cuda")
    st = L.rm_stats()
    g = dLdC.contiguous()
    if hits is not None:
        _check(lib.rm_radio_map_grad_mesh_hits(scene.handle, surface.handle, arr, ntx, C.byref(p), _ptr(g),
                                               _ptr(hits), hits.numel(), _ptr(d_eps), _ptr(d_sig), _ptr(d_tx), sm,
                                               C.byref(st), _ptr(rec), _stream(stream)), "rm_radio_map_grad_mesh_hits")
    else:
        _check(lib.rm_radio_map_grad_mesh(scene.handle, surface.handle, arr, ntx, C.byref(p), _ptr(g), _ptr(d_eps),
                                          _ptr(d_sig), _ptr(d_tx), sm, C.byref(st), _ptr(rec), _stream(stream)),
               "rm_radio_map_grad_mesh")
    out = {"d_eps": d_eps, "d_sigma": d_sig, "d_tx": d_tx, "stats": st.as_dict()}
    if record:
        out["record"] = rec
    return out


def surface(verts, tris, device="cuda", stream=None, builder="auto") -> Scene:
    """A mesh measurement surface: the triangles uploaded with their BVH (one dummy material)."""
    t = np.asarray(tris, np.int32).reshape(-1, 3)
    return Scene(verts, t, np.zeros(len(t), np.int32), np.array([[1.0, 0.0, 0.0]], np.float32), device=device,
                 stream=stream, builder=builder)


def diffraction_map(scene: Scene, txs, params, samples_per_wedge: int, wedges=None, record=False, stream=None,
                    out=None):
    """First-order diffraction maps [ntx, ny, nx] (float32, cuda); add them to trace()'s maps
    for the full radio map.  wedges: (ctypes array, count) or None for all of the scene's."""
    lib = L.load()
    arr, ntx = _tx_array(txs)
    p = params if isinstance(params, L.rm_trace_params) else params_from(params)
    w, nw = wedges if wedges is not None else scene.wedges()
    maps = out if out is not None else torch.empty((ntx, p.ny, p.nx), dtype=torch.float32, device="cuda")
    rec = None
    if record:
        rec = torch.empty((max(ntx * nw * samples_per_wedge, 1), 4), dtype=torch.int32, device="cuda")
    st = L.rm_stats()
    _check(lib.rm_diffraction_map(scene.handle, w, nw, arr, ntx, C.byref(p), int(samples_per_wedge), _ptr(maps),
                                  C.byref(st), _ptr(rec), _stream(stream)), "rm_diffraction_map")
    res = {"maps": maps, "stats": st.as_dict(), "wedges": nw}
    if record:
        res["record"] = rec
    return res


def grad(scene: Scene, txs, params, dLdC: torch.Tensor, sampling=None, record=False, stream=None, hits=None):
    """(d_eps [nm], d_sigma [nm], d_txpos [ntx, 3]) of sum(dLdC * maps), choices frozen, q detached.
    hits: trace(..., keep_hits=True)["hits"] of the same scene, transmitters and params: the
    adjoint then replays the recorded closest hits instead of traversing the BVH."""
    lib = L.load()
    arr, ntx = _tx_array(txs)
    p = params if isinstance(params, L.rm_trace_params) else params_from(params)
    d_eps = torch.zeros(scene.nm, dtype=torch.float32, device="cuda")
    d_sig = torch.zeros(scene.nm, dtype=torch.float32, device="cuda")
    d_tx = torch.zeros((ntx, 3), dtype=torch.float32, device="cuda")
    sm = None if sampling is None else materials(sampling)
    rec = None
    if record:
        nrec = sum(tx_count(arr[i]) for i in range(ntx)) * (p.max_depth + 1)
        rec = torch.empty((max(nrec, 1), 4), dtype=torch.int32, device="cuda")
    st = L.rm_stats()
    g = dLdC.contiguous()
    if hits is not None:
        _check(lib.rm_radio_map_grad_hits(scene.handle, arr, ntx, C.byref(p), _ptr(g), _ptr(hits), hits.numel(),
                                          _ptr(d_eps), _ptr(d_sig), _ptr(d_tx), sm, C.byref(st), _ptr(rec),
                                          _stream(stream)), "rm_radio_map_grad_hits")
    else:
        _check(lib.rm_radio_map_grad(scene.handle, arr, ntx, C.byref(p), _ptr(g), _ptr(d_eps), _ptr(d_sig),
                                     _ptr(d_tx), sm, C.byref(st), _ptr(rec), _stream(stream)), "rm_radio_map_grad")
    out = {"d_eps": d_eps, "d_sigma": d_sig, "d_tx": d_tx, "stats": st.as_dict()}
    if record:
        out["record"] = rec
    return out


def db_mse_loss(maps: torch.Tensor, target: torch.Tensor, floor: float = 1e-15, stream=None):
    """(loss scalar tensor, dL/dmaps, |V|) of the dB mean-squared error over cells above `floor`."""
    lib = L.load()
    m, t = maps.contiguous(), target.contiguous()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    valid = torch.empty(1, dtype=torch.int64, device="cuda")
    g = torch.empty_like(m)
    _check(lib.rm_db_mse_loss(_ptr(m), _ptr(t), m.numel(), float(floor), _ptr(loss), _ptr(g), _ptr(valid),
                              _stream(stream)), "rm_db_mse_loss")
    return loss, g, valid


class TracePlan:
    """A trace captured once into a CUDA graph and replayed with rm_trace_plan_launch."""

    def __init__(self, scene: Scene, txs, params, maps: torch.Tensor, stream=None):
        lib = L.load()
        self._arr, ntx = _tx_array(txs)
        self._p = params if isinstance(params, L.rm_trace_params) else params_from(params)
        self.maps = maps
        self._scene = scene
        h = C.c_void_p()
        _check(lib.rm_trace_plan_create(scene.handle, self._arr, ntx, C.byref(self._p), _ptr(maps), _stream(stream),
                                        C.byref(h)), "rm_trace_plan_create")
        self.handle = h

    def launch(self, stream=None):
        _check(L.load().rm_trace_plan_launch(self.handle, _stream(stream)), "rm_trace_plan_launch")

    def stats(self, stream=None):
        st = L.rm_stats()
        _check(L.load().rm_trace_plan_stats(self.handle, _stream(stream), C.byref(st)), "rm_trace_plan_stats")
        return st.as_dict()

    def free(self):
        if getattr(self, "handle", None):
            L.load().rm_trace_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class RadioMap(torch.autograd.Function):
    """maps = RadioMap.apply(eps_r [nm], sigma [nm], tx_pos [ntx, 3], scene, txs, params, thickness [nm],
    keep_hits=False).

    The forward traces with the given materials and positions; the backward is
    the hand-written adjoint kernel (choices frozen, probabilities detached).
    With keep_hits the forward records every segment's closest-hit leaf (4 bytes
    per ray and depth, held until the backward) and the backward replays them
    instead of traversing the BVH again.
    """

    @staticmethod
    def forward(ctx, eps, sigma, tx_pos, scene, txs, params, thickness, keep_hits=False):
        mats = np.stack([eps.detach().cpu().double().numpy(), sigma.detach().cpu().double().numpy(),
                         np.asarray(thickness, np.float64)], 1)
        scene.set_materials(mats)
        pos = tx_pos.detach().cpu().double().numpy()
        txl = []
        for i, t in enumerate(txs):
            s = t if isinstance(t, L.rm_tx) else tx_from(t)
            s2 = L.rm_tx.from_buffer_copy(s)
            s2._keep = getattr(s, "_keep", None)
            for a in range(3):
                s2.pos[a] = float(pos[i, a])
            txl.append(s2)
        ctx.scene, ctx.txs, ctx.params = scene, txl, params
        ctx.meta = [(t.device, t.dtype) for t in (eps, sigma, tx_pos)]
        f = trace(scene, txl, params, keep_hits=bool(keep_hits))
        ctx.hits = f.get("hits")
        return f["maps"]

    @staticmethod
    def backward(ctx, g):
        r = grad(ctx.scene, ctx.txs, ctx.params, g.contiguous(), hits=ctx.hits)
        ctx.hits = None
        out = [r[k].to(device=d, dtype=t) for k, (d, t) in zip(("d_eps", "d_sigma", "d_tx"), ctx.meta)]
        return out[0], out[1], out[2], None, None, None, None, None
