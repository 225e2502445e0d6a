"""Failure detection without a GPU fault: host-side injection through the C
ABI (rm_debug_inject, RM_FAULT) and a rank that fails on the host before the
sharded path's collective (gloo ranks on CPU; the survivor's collective ends
with an error instead of waiting)."""
import ctypes as C
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2504_21719_b300 import build
    build.build()
    from paper_2504_21719_b300 import _lib
    _lib.load()
    return _lib


def _upload_empty(L):
    """An empty mesh passes validation; the first device call follows."""
    lib = L.load()
    h = C.c_void_p()
    mats = (L.rm_material * 1)(L.rm_material(4.0, 0.01, 0.2))
    return lib.rm_scene_upload(None, 0, None, 0, None, mats, 1, None, C.byref(h)), h


def test_inject_arguments(L):
    lib = L.load()
    assert lib.rm_debug_inject(0, 1) == L.RM_EINVAL
    assert lib.rm_debug_inject(4, 1) == L.RM_EINVAL
    assert lib.rm_debug_inject(L.RM_FAULT_ALLOC, -1) == L.RM_EINVAL
    assert lib.rm_debug_inject(L.RM_FAULT_ALLOC, 0) == L.RM_OK


def test_injected_allocation_failure_is_consumed(L):
    lib = L.load()
    assert lib.rm_debug_inject(L.RM_FAULT_ALLOC, 2) == L.RM_OK
    for _ in range(2):
        st, _h = _upload_empty(L)
        assert st == L.RM_ENOMEM and b"injected" in lib.rm_last_error()
    st, h = _upload_empty(L)          # disarmed: the call proceeds (no device here, or a real upload)
    assert st != L.RM_ENOMEM or b"injected" not in lib.rm_last_error()
    if st == L.RM_OK:
        lib.rm_scene_free(h)


def test_environment_arms_once_per_process():
    code = ("import ctypes as C, sys; sys.path.insert(0, %r)\n"
            "from paper_2504_21719_b300 import _lib as L\n"
            "lib = L.load(); h = C.c_void_p()\n"
            "m = (L.rm_material * 1)(L.rm_material(4.0, 0.01, 0.2))\n"
            "out = []\n"
            "for _ in range(4):\n"
            "    st = lib.rm_scene_upload(None, 0, None, 0, None, m, 1, None, C.byref(h))\n"
            "    out.append(int(st == L.RM_ENOMEM and b'injected' in lib.rm_last_error()))\n"
            "print(''.join(map(str, out)))\n") % ROOT
    env = dict(os.environ, RM_FAULT="alloc:3")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "1110"


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import datetime

    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    from paper_2504_21719_b300.shard import allreduce_maps
    m = torch.ones(16, dtype=torch.float64)
    if rank == 1:
        # a host-side failure between steps: this rank never joins the collective
        raise SystemExit(3)
    try:
        allreduce_maps(m)
        result = "no error"
    except Exception as e:  # the survivor learns of the failure from the collective's timeout
        result = "error: " + type(e).__name__
    with open(out, "w") as f:
        f.write(result)


def test_failed_rank_ends_the_survivors_collective_with_an_error(tmp_path):
    import multiprocessing as mp
    out = str(tmp_path / "r0.txt")
    port = _free_port()
    ctx = mp.get_context("spawn")
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    assert all(not p.is_alive() for p in ps)
    assert ps[1].exitcode == 3
    assert open(out).read().startswith("error")
