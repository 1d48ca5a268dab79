"""The element-partitioned library path (fr_set_comm) on one GPU: two ranks, each a
context on its part of the mesh with one ghost layer, run in two host threads of one
process and exchange ghosts and reductions through host barriers and device-to-device
copies (distributed.LoopbackGroup; no kernel waits on another).

Against one context on the whole mesh:
  - residual, Jacobian-vector product and one FP64 pMG V-cycle: owned parts bit for bit
    (every owned value is computed from the same inputs in the same order; the cycle's
    element-local steps need no exchange and each level's residual exchanges first);
  - FGMRES-based steps (ESDIRK3 at the 1e-12 Newton tolerance, FP64 and mixed
    preconditioner): 1e-10, the converged-step bar (inner products summed in another
    order change only the iteration path);
  - ROS34PW2 at the larger FD step of the ROW parity test: 1e-10;
  - the partitioned context refuses what it does not partition (the network guess, the
    matrix-based coarse smoother, the allocation-free residual)."""
import math
import threading

import numpy as np
import pytest
import torch

from paper_2202_09733_gb300 import api, workloads as w, tableaux as GT
from paper_2202_09733_gb300 import build as B, _native as N
from paper_2202_09733_gb300.distributed import LoopbackGroup, PartitionedContext

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _state(mesh, p, mach=0.3):
    X = w.solution_point_coords(mesh, p)
    s = [np.sin(0.7 * X[0] + 0.4 * X[1] + i) for i in range(4)]
    vel = [math.cos(0.4) + 0.1 * s[1], math.sin(0.4) + 0.1 * s[2]] + ([0.05 * s[3]] if mesh["d"] == 3 else [])
    return np.ascontiguousarray(w.prim_to_cons(1.0 + 0.05 * s[0], vel, (1.0 / (1.4 * mach ** 2)) * (1 + 0.05 * s[3])))


CASES = {
    "vortex_p21": (lambda: w.box2d(6, 6, 10, 10, qg=2, warp=0.1), [2, 1], 0.01),
    "omesh_p32": (lambda: w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3), [3, 2], 0.02),
    "box3d_p21": (lambda: w.box3d(4, 2.0), [2, 1], 0.01),
}


def _run(parts, fn):
    """fn(rank, part) on every rank in its own thread; re-raises the first failure."""
    out, err = [None] * len(parts), [None] * len(parts)

    def work(r):
        try:
            out[r] = fn(r, parts[r])
        except BaseException as ex:              # noqa: BLE001 - reported below
            err[r] = ex
            parts[r].transport.g.bar.abort()
    th = [threading.Thread(target=work, args=(r,)) for r in range(len(parts))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for e in err:
        if e is not None and not isinstance(e, threading.BrokenBarrierError):
            raise e
    for e in err:
        if e is not None:
            raise e
    return out


def _setup(name, nranks=2):
    make, levels, mu = CASES[name]
    mesh = make()
    ph = w.Physics(mu=mu, qinf=w.freestream(mesh["d"], 0.3))
    G = api.fr_create(mesh, ph, levels)
    grp = LoopbackGroup(nranks)
    parts = [PartitionedContext(mesh, ph, levels, r, nranks, grp.transport(r)) for r in range(nranks)]
    return mesh, levels, ph, G, parts


def _gather(parts, xs, shape):
    full = np.zeros(shape)
    for p, x in zip(parts, xs):
        full[:, :, p.loc["owned"]] = p.owned(x).cpu().numpy()
    return full


@pytest.mark.parametrize("name", sorted(CASES))
def test_partitioned_residual_jvp_and_cycle_bitwise(name):
    mesh, levels, ph, G, parts = _setup(name)
    q = _state(mesh, levels[0])
    v = np.random.default_rng(3).standard_normal(q.shape)
    v /= np.linalg.norm(v)
    qd = torch.from_numpy(q).cuda()
    R = api.fr_residual(G, 0, qd)
    Av = api.fr_jvp(G, qd, R, torch.from_numpy(v).cuda(), 1e-6, 2.5)
    dt = 0.3
    c = 1.0 / dt + 1.0 / (0.4358665215084590 * dt)
    api.pmg_setup(G, qd, [2, 2], c, 1.0 / dt)
    Y = api.pmg_precondition(G, qd, R, torch.from_numpy(v).cuda())

    def rank_fn(r, p):
        ql = p.local_state(q)
        vl = p.local_state(v)
        Rl = api.fr_residual(p.ctx, 0, ql)
        Avl = api.fr_jvp(p.ctx, ql, Rl, vl, 1e-6, 2.5)
        api.pmg_setup(p.ctx, ql, [2, 2], c, 1.0 / dt)
        Yl = api.pmg_precondition(p.ctx, ql, Rl, vl)
        torch.cuda.synchronize()
        return Rl, Avl, Yl
    res = _run(parts, rank_fn)
    for k, ref in enumerate((R, Av, Y)):
        got = _gather(parts, [x[k] for x in res], q.shape)
        assert np.array_equal(got, ref.cpu().numpy()), (name, k)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["vortex_p21", "box3d_p21"])
def test_partitioned_esdirk_step(name, precision):
    mesh, levels, ph, G, parts = _setup(name)
    q0 = _state(mesh, levels[0], mach=0.5)
    dt = 10.0 * w.explicit_dt(mesh, levels[0], q0)
    A, b = GT.esdirk3()
    o = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-12,
                       dtau=dt, inv_dtau_star=1.0 / dt, precision=precision, guess="extrap")
    qg = torch.from_numpy(q0.copy()).cuda()
    st = api.esdirk_step(G, A, b, dt, qg, o)
    assert st["converged"]

    def rank_fn(r, p):
        ql = p.local_state(q0)
        s = api.esdirk_step(p.ctx, A, b, dt, ql, o)
        torch.cuda.synchronize()
        return ql, s
    res = _run(parts, rank_fn)
    assert all(s["converged"] for _, s in res)
    assert res[0][1]["n_ptc"] == res[1][1]["n_ptc"]         # one Newton iteration count for all ranks
    got = _gather(parts, [x[0] for x in res], q0.shape)
    ref = qg.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-10
    assert np.abs(got - q0).max() / np.abs(q0).max() > 1e-4


def test_partitioned_row_step():
    mesh, levels, ph, G, parts = _setup("vortex_p21")
    q0 = _state(mesh, levels[0], mach=0.5)
    dt = 10.0 * w.explicit_dt(mesh, levels[0], q0)
    g, a, c, m = GT.ros34pw2()
    o = api.solve_opts(kdim=40, maxit_gmres=400, nsmooth=(2, 2), tol_gmres=1e-12, inv_dtau_star=1.0 / dt, eps=1e-3)
    qg = torch.from_numpy(q0.copy()).cuda()
    api.row_step(G, g, a, c, m, dt, qg, o)

    def rank_fn(r, p):
        ql = p.local_state(q0)
        api.row_step(p.ctx, g, a, c, m, dt, ql, o)
        torch.cuda.synchronize()
        return ql
    res = _run(parts, rank_fn)
    got = _gather(parts, res, q0.shape)
    ref = qg.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-10


def test_partitioned_context_refuses_unpartitioned_features():
    mesh, levels, ph, G, parts = _setup("vortex_p21")
    p = parts[0]
    q = p.local_state(_state(mesh, levels[0]))
    R = torch.empty_like(q)
    rc = N.load().fr_residual_noalloc(p.ctx.handle, 0, api._dev(q), api._dev(R), None)
    assert rc == -1
    with pytest.raises(RuntimeError):
        api.pmg_setup(p.ctx, q, [2, 2], 4.0, 1.0, coarse="mbnk")
