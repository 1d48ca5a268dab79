"""The Weiss-Smith preconditioned Roe flux (fr_physics.flux = 2; Sec. 4.1) on the GPU against
the oracle, on the same seeded inputs, at a moderate and at the low Mach number of the
steady cylinder:
  - the residual on every p-level of the stretched O-mesh (wall and far field, p{4-2-1})
    and of a periodic 3-D box (p{3-2}): bit for bit (the flux follows the oracle's
    evaluation order term by term), and the Jacobian-vector product to 1e-12;
  - one FP64 pMG V-cycle: bit for bit;
  - the FP32 element blocks (element by element, forward mode) against the oracle's FP64
    difference blocks at Ma 0.3: 5e-2 of max |M| (measured 1.5e-2, the same for the
    whole-level colouring; 5e-7 for Roe).  The preconditioned dissipation weighs pressure
    jumps by 1/Ur^2 instead of 1/c^2, and in FP32 a pressure jump is a difference of
    energies rounded to 2^-24 of themselves, so its rounding grows by (c/Ur)^2; at Ma 1e-3
    (c/Ur ~ 1e3, energies ~ 1.8e6 with an FP32 spacing of 0.125 against dynamic pressures
    of 0.5) FP32 cannot carry this flux, which is why the low-Mach steady case keeps the
    FP64 preconditioner with it;
  - a converged ESDIRK3 step of the periodic vortex: 1e-10."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import tableaux as OT
from paper_2202_09733_gb300 import api, workloads as w
from paper_2202_09733_gb300 import build as B, tableaux as GT

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _state(mesh, p, mach):
    X = w.solution_point_coords(mesh, p)
    s = [np.sin(0.6 * X[0] + 0.3 * X[1] + i) for i in range(4)]
    vel = [math.cos(0.3) + 0.1 * s[1], math.sin(0.3) + 0.1 * s[2]] + ([0.05 * s[3]] if mesh["d"] == 3 else [])
    pr = (1.0 / (1.4 * mach ** 2)) * (1 + 0.05 * mach ** 2 * s[3])
    return np.ascontiguousarray(w.prim_to_cons(1.0 + 0.05 * s[0], vel, pr))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def relerr(a, b):
    a = a.cpu().numpy() if torch.is_tensor(a) else a
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = {"omesh_p421": (lambda: w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3), [4, 2, 1]),
         "box3d_p32": (lambda: w.box3d(3, 2.0), [3, 2])}


@pytest.mark.parametrize("mach", [0.3, 1e-3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_jvp_and_cycle(name, mach):
    make, levels = CASES[name]
    mesh = make()
    ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], mach), flux="weiss_smith", ws_umin=1.0)
    O = oracle.Oracle(mesh, ph, levels)
    G = api.fr_create(mesh, ph, levels)
    q = _state(mesh, levels[0], mach)
    ql = q
    for l in range(len(levels)):
        if l:
            ql = O.restrict(ql, l - 1)
        R_or = O.residual(ql, l)
        R = api.fr_residual(G, l, dev(ql))
        assert np.array_equal(R.cpu().numpy(), R_or), (name, mach, l)
    Rq = O.residual(q)
    v = np.random.default_rng(4).standard_normal(q.shape)
    v /= np.linalg.norm(v)
    assert relerr(api.fr_jvp(G, dev(q), dev(Rq), dev(v), 1e-6, 3.0), O.jvp(q, Rq, v, 1e-6, 3.0)) <= 1e-12
    if mesh["E"] <= 128:
        dt = 0.05
        c = 1.0 / dt + 1.0 / (0.4358665215084590 * dt)
        nsm = [2, 2, 5][:len(levels)]
        O.pmg_setup(q, nsm, c, 1.0 / dt)
        api.pmg_setup(G, dev(q), nsm, c, 1.0 / dt)
        X = np.random.default_rng(5).standard_normal(q.shape)
        Y = api.pmg_precondition(G, dev(q), dev(Rq), dev(X))
        assert np.array_equal(Y.cpu().numpy(), O.pmg_apply(q, Rq, X)), (name, mach)


@pytest.mark.parametrize("mach,tol", [(0.3, 5e-2)])
def test_fp32_blocks(mach, tol):
    # |u| = 1 +- 0.1 here: the floor 0.5 keeps Ur = |u| away from the kink of
    # max(|u|, umin), where one-sided derivatives and differences across it disagree
    mesh = w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3)
    ph = w.Physics(mu=0.02, qinf=w.freestream(2, mach), flux="weiss_smith", ws_umin=0.5)
    O = oracle.Oracle(mesh, ph, [3])
    G = api.fr_create(mesh, ph, [3])
    q = _state(mesh, 3, mach)
    shift = 4.2 / mach
    M = api.fr_elem_blocks_f32(G, 0, torch.from_numpy(q.astype(np.float32)).cuda(), shift, "local")
    M_or = torch.from_numpy(O.elem_blocks(q, shift, np.arange(mesh["E"]))).transpose(1, 2).cuda()
    err = (M.double() - M_or).abs().max().item() / M_or.abs().max().item()
    assert err <= tol, err


def test_esdirk_step_converged_state():
    mesh = w.box2d(4, 4, 10, 10, qg=2, warp=0.1)
    mach = 0.1
    ph = w.Physics(mu=0.01, qinf=w.freestream(2, mach), flux="weiss_smith", ws_umin=0.5)
    X = w.solution_point_coords(mesh, 2)
    q0 = np.ascontiguousarray(w.isentropic_vortex(X, 5, 5, 5.0, mach, 10, 10))
    dt = 10.0 * w.explicit_dt(mesh, 2, q0)
    O = oracle.Oracle(mesh, ph, [2, 1])
    G = api.fr_create(mesh, ph, [2, 1])
    A, b, _ = OT.esdirk3()
    oo = O.opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-12, dtau=dt,
                inv_dtau_star=1.0 / dt)
    q_or, st_or = O.esdirk_step(A, b, dt, q0, oo)
    Ag, bg = GT.esdirk3()
    go = api.solve_opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-12,
                        dtau=dt, inv_dtau_star=1.0 / dt)
    qg = dev(q0)
    st = api.esdirk_step(G, Ag, bg, dt, qg, go)
    assert st_or["converged"] and st["converged"]
    assert relerr(qg, q_or) <= 1e-10
    assert relerr(qg, q0) > 1e-6
