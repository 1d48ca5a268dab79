"""Failure detection on the GPU by host-side fault injection (no device fault, trap or
hang): a NaN written into the state, an unreachable tolerance and a zero right-hand side
come back as status codes (FR_ERR_NONFINITE, FR_ERR_NOT_CONVERGED, a clean zero solve),
the context stays usable afterwards, and the retrying driver turns a step that failed
on corrupted input into two half steps from the restored state."""
import math

import numpy as np
import pytest
import torch

from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B
from paper_2202_09733_gb300 import tableaux as GT
from paper_2202_09733_gb300 import _native as N
from paper_2202_09733_gb300 import steplog as S

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module")
def vortex():
    B.build()
    mesh = w.box2d(4, 4, 10, 10, qg=2, warp=0.1)
    ph = w.Physics(mu=0.01, qinf=w.freestream(2, 0.5))
    X = w.solution_point_coords(mesh, 2)
    q0 = np.ascontiguousarray(w.isentropic_vortex(X, 5, 5, 5.0, 0.5, 10, 10))
    dt = 10.0 * w.explicit_dt(mesh, 2, q0)
    G = api.fr_create(mesh, ph, [2, 1])
    return G, q0, dt


def opts(dt, **kw):
    base = dict(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-10, dtau=dt,
                inv_dtau_star=1.0 / dt)
    base.update(kw)
    return api.solve_opts(**base)


def test_nan_state_is_reported_and_the_context_recovers(vortex):
    G, q0, dt = vortex
    A, b = GT.esdirk3()
    q = torch.from_numpy(q0.copy()).cuda()
    q[1, 3, 5] = float("nan")
    with pytest.raises(N.FrError) as ex:
        api.esdirk_step(G, A, b, dt, q, opts(dt))
    assert ex.value.code == -5
    q = torch.from_numpy(q0.copy()).cuda()
    st = api.esdirk_step(G, A, b, dt, q, opts(dt))
    assert st["converged"] and torch.isfinite(q).all()


def test_unreachable_tolerance_is_not_converged(vortex):
    G, q0, dt = vortex
    A, b = GT.esdirk3()
    q = torch.from_numpy(q0.copy()).cuda()
    st = api.esdirk_step(G, A, b, dt, q, opts(dt, tol_newton=0.0, max_ptc=2))
    assert not st["converged"] and st["n_ptc"] == 2 * (len(b) - 1)
    with pytest.raises(N.FrError) as ex:
        api.esdirk_step(G, A, b, dt, torch.from_numpy(q0.copy()).cuda(), opts(dt, tol_newton=0.0, max_ptc=2),
                        allow_not_converged=False)
    assert ex.value.code == -4


def test_zero_right_hand_side(vortex):
    G, q0, dt = vortex
    q = torch.from_numpy(q0.copy()).cuda()
    R = api.fr_residual(G, 0, q)
    x, st = api.gmres_solve(G, q, R, torch.zeros_like(q), kdim=10, maxit=10, tol=1e-6, shift=1.0 / dt)
    assert st["iters"] == 0 and bool((x == 0).all())


def test_retrying_driver_restores_and_halves(vortex):
    G, q0, dt = vortex
    A, b = GT.esdirk3()
    corrupt = [True]

    def step(q, h):
        if corrupt[0]:
            corrupt[0] = False
            q[0, 0, 0] = float("nan")           # injected fault: this attempt must fail
        return api.esdirk_step(G, A, b, h, q, opts(dt))

    q = torch.from_numpy(q0.copy()).cuda()
    t = S.march(step, q, 0.0, dt, 1, sync=torch.cuda.synchronize)
    assert t == dt and torch.isfinite(q).all()
    ref = torch.from_numpy(q0.copy()).cuda()
    for _ in range(2):
        api.esdirk_step(G, A, b, 0.5 * dt, ref, opts(dt))
    assert float((q - ref).abs().max() / ref.abs().max()) <= 1e-9


def test_failed_step_leaves_the_guess_history_unchanged(vortex):
    """A step that does not converge must not enter the learned guess's history, and a
    retry at dt/2 must not extrapolate from states spaced by dt: a context that saw the
    failed attempt and one that never did take the same (bit for bit) steps afterwards."""
    _, q0, dt = vortex
    mesh = w.box2d(4, 4, 10, 10, qg=2, warp=0.1)
    ph = w.Physics(mu=0.01, qinf=w.freestream(2, 0.5))
    A, b = GT.esdirk3()
    GA, GB = api.fr_create(mesh, ph, [2, 1]), api.fr_create(mesh, ph, [2, 1])
    qa, qb = torch.from_numpy(q0.copy()).cuda(), torch.from_numpy(q0.copy()).cuda()
    for _ in range(3):
        api.esdirk_step(GA, A, b, dt, qa, opts(dt, guess="extrap"))
        api.esdirk_step(GB, A, b, dt, qb, opts(dt, guess="extrap"))
    before = api.fr_checkpoint_save(GA)
    qf = qa.clone()
    st = api.esdirk_step(GA, A, b, dt, qf, opts(dt, guess="extrap", tol_newton=0.0, max_ptc=1))
    assert not st["converged"]
    assert api.fr_checkpoint_save(GA) == before           # history and ring untouched
    picks = []
    for G, q in ((GA, qa), (GB, qb)):
        ps = []
        for h in (0.5 * dt,) * 4:
            s = api.esdirk_step(G, A, b, h, q, opts(dt, guess="extrap"))
            assert s["converged"]
            ps.append(tuple(s["guess_pick"]))
        picks.append(ps)
    assert picks[0] == picks[1]
    # a changed dt restarts the history: the first two half steps have no extrapolation
    # candidate, the later ones do (three states spaced by dt/2)
    assert sum(picks[0][0]) == sum(picks[0][1]) == 0 and sum(picks[0][3]) > 0
    assert torch.equal(qa, qb)
