"""Pins of the oracle's FR residual R(q) (Eq. 1 with R = -div f; Sec. 2.1).

  - free-stream preservation to round-off on curved, jittered and stretched meshes, on
    every p-level (including levels whose geometry is re-interpolated to degree p);
  - discrete conservation: sum_e sum_i w_i J_i R_i = 0 on periodic meshes;
  - order of accuracy against manufactured solutions differentiated by sympy
    (inviscid order p, viscous part order >= p-1), 2-D curved and 3-D;
  - linear stability: the linearised operator about a rest state has no eigenvalue with a
    positive real part beyond finite-difference noise;
  - bitwise consistency of the element-local residual with the full residual;
  - the viscous part linearised about rest: mass-symmetric (affine) and negative
    semidefinite (affine and curved)."""
import math

import numpy as np
import pytest

import oracle
from paper_2202_09733_gb300 import workloads as w
import mms


def _uniform(O, l, qinf):
    return np.broadcast_to(qinf[:, None, None], O.shape(l)).copy()


def _flux_scale(qinf, d, h):
    rho, vel = qinf[0], qinf[1:1 + d] / qinf[0]
    p = 0.4 * (qinf[d + 1] - 0.5 * rho * np.dot(vel, vel))
    return (qinf[d + 1] + p) * max(1.0, np.abs(vel).max()) * 2.0 / h


@pytest.mark.parametrize("warp", [0.0, 0.15])
def test_freestream_box2d(warp):
    mesh = w.box2d(4, 3, 10, 7.5, qg=2, warp=warp)
    qinf = w.freestream(2, 0.3, aoa=0.4)
    O = oracle.Oracle(mesh, w.Physics(mu=0.02, qinf=qinf), [4, 3, 2, 1])
    for l, p in enumerate(O.levels):
        R = O.residual(_uniform(O, l, qinf), l)
        assert np.abs(R).max() <= 1e-14 * _flux_scale(qinf, 2, mesh["h_min"]) * (p + 1) ** 2


def test_freestream_omesh_all_levels():
    mesh = w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3)
    f = mesh["faces"].copy()
    f[f[:, 5] == 2, 5] = 1          # far field on both boundaries: the free stream is exact
    mesh["faces"] = f
    qinf = w.freestream(2, 0.3)
    O = oracle.Oracle(mesh, w.Physics(mu=0.01, qinf=qinf), [4, 2, 1])
    for l, p in enumerate(O.levels):
        R = O.residual(_uniform(O, l, qinf), l)
        assert np.abs(R).max() <= 1e-14 * _flux_scale(qinf, 2, mesh["h_min"]) * (p + 1) ** 2
        assert O.jacobian_det(l).min() > 0


def test_freestream_box3d():
    mesh = w.box3d(3, 2.0)
    qinf = w.freestream(3, 0.2)
    qinf[2], qinf[3] = 0.3, -0.2
    qinf[4] += 0.5 * (0.09 + 0.04)
    O = oracle.Oracle(mesh, w.Physics(mu=0.01, qinf=qinf), [3, 2])
    for l, p in enumerate(O.levels):
        R = O.residual(_uniform(O, l, qinf), l)
        assert np.abs(R).max() <= 1e-14 * _flux_scale(qinf, 3, mesh["h_min"]) * (p + 1) ** 2


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_conservation_periodic(p):
    mesh = w.box2d(5, 4, 10, 8, qg=2, warp=0.15)
    O = oracle.Oracle(mesh, w.Physics(mu=0.05, qinf=w.freestream(2, 0.5)), [p])
    X = w.solution_point_coords(mesh, p)
    q = w.isentropic_vortex(X, 5, 4, 5.0, 0.5, 10, 8)
    R = O.residual(q)
    J = O.jacobian_det()
    t = oracle.table(p)
    W = np.outer(t["w"], t["w"]).ravel()
    tot = np.einsum("i,ie,vie->v", W, J, R)
    scale = np.einsum("i,ie,vie->v", W, J, np.abs(R))
    assert np.all(np.abs(tot) <= 1e-13 * scale)


def test_conservation_periodic_3d():
    mesh = w.box3d(3, 2 * math.pi)
    state, _ = mms.exact_rhs(3, 0.05)
    O = oracle.Oracle(mesh, w.Physics(mu=0.05, qinf=np.zeros(5)), [2])
    X = w.solution_point_coords(mesh, 2)
    R = O.residual(state(X))
    J = O.jacobian_det()
    t = oracle.table(2)
    W = np.einsum("i,j,k->kji", t["w"], t["w"], t["w"]).ravel()
    tot = np.einsum("i,ie,vie->v", W, J, R)
    scale = np.einsum("i,ie,vie->v", W, J, np.abs(R))
    assert np.all(np.abs(tot) <= 1e-13 * scale)


def _mms_errors(d, p, ns, mu_split):
    s1, t1 = mms.exact_rhs(d, 0.05)
    s0, t0 = mms.exact_rhs(d, 0.0)
    errs = []
    for n in ns:
        mesh = w.box2d(n, n, 2 * math.pi, 2 * math.pi, qg=2, warp=0.1) if d == 2 else w.box3d(n, 2 * math.pi)
        X = w.solution_point_coords(mesh, p)
        if mu_split:
            Ra = oracle.Oracle(mesh, w.Physics(mu=0.05, qinf=np.zeros(d + 2)), [p]).residual(s1(X))
            Rb = oracle.Oracle(mesh, w.Physics(mu=0.0, qinf=np.zeros(d + 2)), [p]).residual(s1(X))
            tv = t1(X) - t0(X)
            errs.append(np.sqrt(np.mean(((Ra - Rb) - tv) ** 2)) / np.sqrt(np.mean(tv ** 2)))
        else:
            R = oracle.Oracle(mesh, w.Physics(mu=0.0, qinf=np.zeros(d + 2)), [p]).residual(s0(X))
            errs.append(np.sqrt(np.mean((R - t0(X)) ** 2)))
    errs = np.array(errs)
    return errs, np.log2(errs[:-1] / errs[1:])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_order_inviscid_curved_2d(p):
    errs, rates = _mms_errors(2, p, [4, 8, 16], False)
    assert rates[-1] >= p - 0.2


@pytest.mark.parametrize("p", [2, 3, 4])
def test_order_viscous_part_curved_2d(p):
    errs, rates = _mms_errors(2, p, [4, 8, 16], True)
    assert rates[-1] >= p - 1 - 0.25
    assert errs[-1] < 0.06


def test_order_3d():
    errs, rates = _mms_errors(3, 3, [3, 6], False)
    assert rates[-1] >= 3 - 0.3
    errs, rates = _mms_errors(3, 3, [3, 6], True)
    assert rates[-1] >= 2 - 0.25


@pytest.mark.parametrize("p", [1, 2, 3])
def test_linearised_operator_is_stable(p):
    mesh = w.box2d(3, 3, 3.0, 3.0, qg=2, warp=0.1)
    qinf = w.freestream(2, 0.3)
    qinf[1] = 0.0
    qinf[3] = (1 / (1.4 * 0.09)) / 0.4
    O = oracle.Oracle(mesh, w.Physics(mu=0.2, qinf=qinf), [p])
    q = _uniform(O, 0, qinf)
    R0 = O.residual(q).ravel()
    N = q.size
    J = np.zeros((N, N))
    for j in range(N):
        qq = q.ravel().copy()
        qq[j] += 1e-6
        J[:, j] = (O.residual(qq.reshape(q.shape)).ravel() - R0) / 1e-6
    ev = np.linalg.eigvals(J)
    assert ev.real.max() <= 1e-7 * np.abs(ev).max()


def test_element_residual_matches_full_residual():
    mesh = w.omesh(4, 6, 0.5, 3.0, 0.05, jitter=0.05, seed=5)
    wl = w.Physics(mu=0.05, qinf=w.freestream(2, 0.4))
    O = oracle.Oracle(mesh, wl, [3])
    X = w.solution_point_coords(mesh, 3)
    rng = np.random.default_rng(0)
    q = w.prim_to_cons(1 + 0.1 * np.sin(X[0]), [1 + 0.1 * np.cos(X[1]), 0.1 * np.sin(X[0] * X[1])],
                       w.freestream(2, 0.4)[3] * 0.4 * np.ones_like(X[0]))
    q = np.ascontiguousarray(q)
    for e in [0, 5, 13, 23]:
        qe = q[:, :, e] + 1e-3 * rng.standard_normal(q[:, :, e].shape)
        O.residual(q)
        Re = O.elem_residual(q, e, qe)
        qq = q.copy()
        qq[:, :, e] = qe
        Rfull = O.residual(qq)
        assert np.array_equal(Re, Rfull[:, :, e])


@pytest.mark.parametrize("warp,p", [(0.0, 1), (0.0, 2), (0.1, 1), (0.1, 2)])
def test_br2_viscous_operator_at_rest(warp, p):
    """The viscous part of R linearised about a uniform rest state, momentum rows and
    columns (the vector Laplacian of the stress), weighted by the Gauss-Legendre mass
    matrix w_i J_i: symmetric to finite-difference accuracy on affine quads (BR2 is a
    symmetric primal scheme) and negative semidefinite; on curved quads (metric terms
    collocated, not integrated exactly) only its symmetric part is required to be
    negative semidefinite."""
    mesh = w.box2d(3, 3, 3.0, 3.0, qg=2, warp=warp)
    q0 = np.array([1.0, 0.0, 0.0, (1 / (1.4 * 0.09)) / 0.4])

    def jac(mu):
        O = oracle.Oracle(mesh, w.Physics(mu=mu, qinf=q0.copy()), [p])
        q = _uniform(O, 0, q0)
        N = q.size
        J = np.zeros((N, N))
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1e-6
            J[:, j] = (O.residual(q + e.reshape(q.shape)) - O.residual(q - e.reshape(q.shape))).ravel() / 2e-6
        return J, O

    J1, O = jac(0.1)
    J0, _ = jac(0.0)
    Np, E = (p + 1) ** 2, mesh["E"]
    t = oracle.table(p)
    Wm = (np.outer(t["w"], t["w"]).ravel()[:, None] * O.jacobian_det()).ravel()
    idx = np.concatenate([v * Np * E + np.arange(Np * E) for v in (1, 2)])
    S = np.concatenate([Wm, Wm])[:, None] * (J1 - J0)[np.ix_(idx, idx)]
    scale = np.abs(S).max()
    if warp == 0.0:
        assert np.abs(S - S.T).max() <= 1e-7 * scale
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).max() <= 1e-8 * scale
