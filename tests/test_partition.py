"""Element partition (partition.py, distributed.py) on the CPU.

Single process: the recursive bisection covers every element once with balanced parts;
each local mesh holds its owned elements and exactly the face neighbours of them as
ghosts; the exchange plan sends every ghost's owner copy.

Two gloo ranks (torch.distributed on the host): each rank fills its ghosts through the
transport the GPU path uses (TorchDistTransport) in the library's exchange layout, then
evaluates the oracle's residual and Jacobian-vector product on its local mesh.  The owned
parts equal the single-domain results bit for bit (an element's residual depends on its
own and its face neighbours' states only), and the owned inner products summed over the
ranks equal the single-domain ones to round-off (another summation order)."""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2202_09733_gb300 import partition as PT, workloads as w   # noqa: E402


def _meshes():
    return {"omesh": (w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3), [3, 2]),
            "box3d": (w.box3d(4, 2.0), [2, 1]),
            "vortex": (w.box2d(6, 6, 10, 10, qg=2, warp=0.1), [2, 1])}


@pytest.mark.parametrize("name", ["omesh", "box3d", "vortex"])
@pytest.mark.parametrize("nranks", [2, 3])
def test_partition_ghost_layer_and_plan(name, nranks):
    mesh, _ = _meshes()[name]
    owner = PT.partition(mesh, nranks)
    counts = np.bincount(owner, minlength=nranks)
    assert counts.sum() == mesh["E"] and counts.max() - counts.min() <= nranks
    locs = [PT.local_problem(mesh, owner, r) for r in range(nranks)]
    plans = PT.exchange_plan(owner, locs)
    faces = np.asarray(mesh["faces"])
    for r, loc in enumerate(locs):
        own = set(loc["owned"].tolist())
        nb = set()
        for a, fa, b, fb, o, bc in faces:
            if b >= 0 and (a in own) != (b in own):
                nb.add(int(b) if a in own else int(a))
        assert set(loc["ghosts"].tolist()) == nb
        assert loc["mesh"]["E"] == len(own) + len(nb)
        # every element face of the local mesh appears exactly once
        lf = loc["mesh"]["faces"]
        seen = {}
        for a, fa, b, fb, o, bc in lf:
            for e, f in ((a, fa), (b, fb)):
                if e >= 0:
                    seen[(int(e), int(f))] = seen.get((int(e), int(f)), 0) + 1
        assert len(seen) == loc["mesh"]["E"] * 2 * mesh["d"] and max(seen.values()) == 1
        # what r receives from p is what p sends to r
        for p in range(nranks):
            assert plans[p]["send_counts"][r] == plans[r]["recv_counts"][p]
            sent = locs[p]["owned"][plans[p]["send"][r]]
            assert np.array_equal(sent, loc["ghosts"][loc["ghost_owner"] == p])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, name, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        from paper_2202_09733_gb300.distributed import TorchDistTransport
        oracle.set_threads(1)
        mesh, levels = _meshes()[name]
        ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], 0.3))
        X = w.solution_point_coords(mesh, levels[0])
        rng = np.random.default_rng(1)
        rho = 1.0 + 0.05 * np.sin(0.7 * X[0] + 0.2)
        vel = [0.9 + 0.1 * np.cos(0.5 * X[1]), 0.3 + 0.05 * np.sin(X[0])] + ([0.05 * np.cos(X[2])] if mesh["d"] == 3 else [])
        q = np.ascontiguousarray(w.prim_to_cons(rho, vel, (1.0 / (1.4 * 0.09)) * (1 + 0.05 * np.cos(X[1]))))
        v = rng.standard_normal(q.shape)
        v /= np.linalg.norm(v)
        owner = PT.partition(mesh, ws)
        locs = [PT.local_problem(mesh, owner, r) for r in range(ws)]
        plan = PT.exchange_plan(owner, locs)[rank]
        loc = locs[rank]
        T = TorchDistTransport()

        def fill_ghosts(x_global):
            x = PT.scatter_state(x_global, loc).copy()
            x[:, :, loc["n_owned"]:] = np.nan                 # only the exchange may fill them
            idx = np.concatenate(plan["send"]).astype(np.int64)
            send = torch.from_numpy(PT.pack_owned(x, idx).copy())
            eb = x.shape[0] * x.shape[1] * 8
            nrecv = x.shape[2] - loc["n_owned"]
            recv = torch.zeros(nrecv * eb, dtype=torch.uint8)
            T.exchange(send, recv, [c * eb for c in plan["send_counts"]], [c * eb for c in plan["recv_counts"]])
            PT.unpack_ghosts(x, recv.numpy(), loc["n_owned"])
            return x

        ql = fill_ghosts(q)
        ghosts_ok = bool(np.array_equal(ql, PT.scatter_state(q, loc)))
        O = oracle.Oracle(loc["mesh"], ph, levels)
        Rl = O.residual(ql)
        eps = 1e-6
        ql_p = fill_ghosts(q + eps * v)                     # the state the product perturbs
        Rp = O.residual(ql_p)
        n = loc["n_owned"]
        Av_owned = (2.0 * v[:, :, loc["owned"]] - (Rp[:, :, :n] - Rl[:, :, :n]) / eps)
        dots = np.array([np.sum(Rl[:, :, :n] * Rl[:, :, :n]), np.sum(v[:, :, loc["owned"]] * Rl[:, :, :n])])
        T.allreduce(dots, 0)
        out[rank] = dict(ghosts_ok=ghosts_ok, owned=loc["owned"], R=Rl[:, :, :n], Av=Av_owned, dots=dots)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["omesh", "box3d"])
def test_two_gloo_ranks_match_single_domain(name):
    import oracle
    mesh, levels = _meshes()[name]
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, name, out), nprocs=2, join=True)
    ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], 0.3))
    X = w.solution_point_coords(mesh, levels[0])
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.05 * np.sin(0.7 * X[0] + 0.2)
    vel = [0.9 + 0.1 * np.cos(0.5 * X[1]), 0.3 + 0.05 * np.sin(X[0])] + ([0.05 * np.cos(X[2])] if mesh["d"] == 3 else [])
    q = np.ascontiguousarray(w.prim_to_cons(rho, vel, (1.0 / (1.4 * 0.09)) * (1 + 0.05 * np.cos(X[1]))))
    v = rng.standard_normal(q.shape)
    v /= np.linalg.norm(v)
    O = oracle.Oracle(mesh, ph, levels)
    R = O.residual(q)
    Av = O.jvp(q, R, v, 1e-6, 2.0)
    for r in range(2):
        o = out[r]
        assert o["ghosts_ok"]
        assert np.array_equal(o["R"], R[:, :, o["owned"]])
        assert np.array_equal(o["Av"], Av[:, :, o["owned"]])
        assert np.allclose(o["dots"], [np.sum(R * R), np.sum(v * R)], rtol=1e-13, atol=0)
