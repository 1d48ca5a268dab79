"""fr_residual_noalloc: the residual for callers that cannot allocate device memory when
they call it (code under CUDA stream capture in the global mode, hosts whose device
memory belongs to another allocator with a fixed budget, real-time loops that must not
pay for or risk an allocation).  It must give exactly what fr_residual gives, call after
call, without allocating, and refuse meshes whose stage scratch exceeds its fixed
16 MiB device array.  Collected last so that a run stopping at the first failure has
run everything else first."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B, _native as N

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module")
def lib():
    """The library, after the documented first call on this device: that call looks up the
    array's device address (which may load the library's device module and with it the
    array); every later call must leave the device's free memory unchanged."""
    B.build()
    L = N.load()
    mesh = w.box2d(2, 2, 10, 10, qg=2)
    ctx = api.fr_create(mesh, w.Physics(mu=0.01, qinf=w.freestream(2, 0.3)), [1])
    q = torch.from_numpy(_state(mesh, 1)).cuda()
    R = torch.empty_like(q)
    rc = L.fr_residual_noalloc(ctx.handle, 0, C.c_void_p(q.data_ptr()), C.c_void_p(R.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.fr_last_error()
    torch.cuda.synchronize()
    return L


def _state(mesh, p, mach=0.3):
    X = w.solution_point_coords(mesh, p)
    s = [np.sin(0.7 * X[0] + 0.4 * X[1] + i) for i in range(4)]
    vel = [1.0 + 0.1 * s[1], 0.3 + 0.1 * s[2]] + ([0.05 * s[3]] if mesh["d"] == 3 else [])
    return np.ascontiguousarray(w.prim_to_cons(1.0 + 0.05 * s[0], vel, (1.0 / (1.4 * mach ** 2)) * (1 + 0.05 * s[3])))


@pytest.mark.parametrize("which", ["vortex2d", "box3d"])
def test_noalloc_matches_fr_residual_twice(lib, which):
    if which == "vortex2d":
        mesh, levels = w.box2d(8, 8, 10, 10, qg=2, warp=0.1), [2, 1]
    else:
        mesh, levels = w.box3d(3, 2 * math.pi), [3, 2]
    ph = w.Physics(mu=0.01, qinf=w.freestream(mesh["d"], 0.3))
    ctx = api.fr_create(mesh, ph, levels)
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    for level in range(len(levels)):
        q = torch.from_numpy(_state(mesh, levels[level])).cuda()
        ref = api.fr_residual(ctx, level, q)
        outs = [torch.full_like(q, float("nan")) for _ in range(2)]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for R in outs:   # two calls in a row share (and reuse) the same device array
            rc = lib.fr_residual_noalloc(ctx.handle, level, C.c_void_p(q.data_ptr()), C.c_void_p(R.data_ptr()), sp)
            assert rc == 0, lib.fr_last_error()
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
        for R in outs:
            err = (R - ref).abs().max().item() / ref.abs().max().item()
            assert err <= 1e-12
            assert torch.equal(R, ref)


def test_noalloc_rejects_levels_beyond_the_array(lib):
    mesh = w.omesh(64, 128, 0.5, 20.0, 2e-4, jitter=0.0)
    ph = w.Physics(mu=0.01, qinf=w.freestream(2, 0.3))
    ctx = api.fr_create(mesh, ph, [4])
    q = torch.ones((4, 25, mesh["E"]), dtype=torch.float64, device="cuda")
    R = torch.empty_like(q)
    rc = lib.fr_residual_noalloc(ctx.handle, 0, C.c_void_p(q.data_ptr()), C.c_void_p(R.data_ptr()),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"16 MiB" in lib.fr_last_error()
