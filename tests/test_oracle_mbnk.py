"""Pins of the oracle's matrix-based Newton-Krylov (MBNK) smoother of the coarsest level
(Sec. 3.2: GMRES of at most 5 iterations to a relative tolerance of 1e-1 on the assembled
linearised operator; block-Jacobi stands in for the per-block ILU0 the paper uses under
domain decomposition, the whole level being one block here):

  neighbour table   every interior face listed from both sides; faces reaching an element
                    twice (periodic mesh two elements wide) listed once;
  assembled A       A x = shift x - J x for the central-difference Jacobian J of the
                    level's residual (random and single-element x), on a curved O-mesh
                    with wall and far-field faces, a two-wide periodic box and hexes;
  GMRES             one iteration is the minimal-residual step along Md^-1 r (closed
                    form); enough iterations give numpy's dense solve; the stopping rule
                    takes the first iteration whose residual meets the tolerance, and the
                    returned estimate is the true residual;
  pMG with MBNK     a one-level cycle with one exact MBNK step is (c I - J)^-1 X; a
                    two-level cycle with MBNK at the bottom keeps the fixed point
                    (c I - J)^-1 X; an ESDIRK3 step converges to the same state as with
                    element-Jacobi smoothing."""
import math

import numpy as np
import pytest

import oracle
from oracle import tableaux as TB
from paper_2202_09733_gb300 import workloads as w
from smooth_state import angled_flow


def wavy(mesh, p, seed=0):
    X = w.solution_point_coords(mesh, p)
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.3, 1.2, size=(4, mesh["d"]))
    s = [np.sin(sum(k[i, c] * X[c] for c in range(mesh["d"])) + i) for i in range(4)]
    vel = [math.cos(0.4) + 0.1 * s[1], math.sin(0.4) + 0.1 * s[2]] + ([0.05 * s[3]] if mesh["d"] == 3 else [])
    return np.ascontiguousarray(w.prim_to_cons(1.0 + 0.05 * s[0], vel, (1.0 / (1.4 * 0.09)) * (1 + 0.05 * s[3])))


MESHES = {
    "omesh": lambda: (w.omesh(4, 6, 0.5, 3.0, 0.05, jitter=0.05, seed=5), [2, 1]),
    "box2d_two_wide": lambda: (w.box2d(2, 3, 4.0, 6.0, qg=2, warp=0.1), [2, 1]),
    "box3d": lambda: (w.box3d(3, 2.0), [2, 1]),
}


@pytest.fixture(scope="module", params=sorted(MESHES))
def lvl(request):
    mesh, levels = MESHES[request.param]()
    ph = w.Physics(mu=0.02, qinf=w.freestream(mesh["d"], 0.3))
    O = oracle.Oracle(mesh, ph, levels)
    q = wavy(mesh, levels[0])
    c, ids = 3.0, 1.5
    O.pmg_setup(q, [1, 1], c, ids, coarse="mbnk")
    qc = O.restrict(q, 0)
    return dict(name=request.param, mesh=mesh, O=O, q=q, qc=qc, shift=c + ids, l=1)


def test_neighbour_table(lvl):
    O, mesh = lvl["O"], lvl["mesh"]
    nbr = O.neighbours()
    E, nf = nbr.shape
    for eL, fL, eR, fR, orient, bc in mesh["faces"]:
        if eR < 0:
            assert nbr[eL, fL] == -1
        else:
            assert nbr[eL, fL] in (eR, -1) and nbr[eR, fR] in (eL, -1)
            assert eR in nbr[eL] and eL in nbr[eR]
    for e in range(E):
        got = [n for n in nbr[e] if n >= 0]
        assert len(got) == len(set(got)) and e not in got
    if lvl["name"] == "box2d_two_wide":
        assert (nbr >= 0).sum(axis=1).max() == 3          # the x-neighbour is reached twice, listed once


def _jac_dir(O, qc, x, l, h=1e-6):
    s = h / max(np.abs(x).max(), 1e-300)
    return (O.residual(qc + s * x, l) - O.residual(qc - s * x, l)) / (2 * s)


def test_assembled_operator_is_the_jacobian(lvl):
    O, qc, l, shift = lvl["O"], lvl["qc"], lvl["l"], lvl["shift"]
    rng = np.random.default_rng(1)
    xs = [rng.standard_normal(qc.shape) for _ in range(3)]
    one = np.zeros(qc.shape)
    one[:, :, 1] = rng.standard_normal(qc.shape[:2])        # a single element's dofs
    xs.append(one)
    for x in xs:
        Ax = O.mbnk_matvec(x, l)
        ref = shift * x - _jac_dir(O, qc, x, l)
        assert np.abs(Ax - ref).max() <= 1e-6 * np.abs(ref).max()
    # the single-element vector touches that element and its face neighbours only
    Ax = O.mbnk_matvec(one, l)
    touched = set(np.nonzero(np.abs(Ax).sum(axis=(0, 1)))[0])
    assert touched <= {1} | set(O.neighbours()[1][O.neighbours()[1] >= 0])


def test_nbr_blocks_match_assembled_operator(lvl):
    O, qc, l, shift = lvl["O"], lvl["qc"], lvl["l"], lvl["shift"]
    Ob = O.nbr_blocks(qc, l)
    nbr = O.neighbours()
    nd = Ob.shape[2]
    E = qc.shape[2]
    e = E // 2
    for f in range(nbr.shape[1]):
        n = nbr[e, f]
        if n < 0:
            assert not Ob[e, f].any()
            continue
        for j in range(nd):
            x = np.zeros(qc.shape)
            x.reshape(nd, E)[j, n] = 1.0
            col = O.mbnk_matvec(x, l).reshape(nd, E)[:, e]
            assert np.array_equal(col, Ob[e, f][:, j])


def test_one_iteration_is_the_minimal_residual_step(lvl):
    O, q, qc, l, shift = lvl["O"], lvl["q"], lvl["qc"], lvl["l"], lvl["shift"]
    O.pmg_setup(q, [1, 1], 3.0, 1.5, coarse="mbnk", mbnk_maxit=1, mbnk_tol=0.0)
    r = np.random.default_rng(2).standard_normal(qc.shape)
    d, k, rel = O.mbnk_solve(r, l)
    z = O.block_solve(r, l)
    Az = O.mbnk_matvec(z, l)
    alpha = np.vdot(r, Az) / np.vdot(Az, Az)
    assert k == 1
    assert np.abs(d - alpha * z).max() <= 1e-12 * np.abs(alpha * z).max()
    assert abs(rel - np.linalg.norm(r - alpha * Az) / np.linalg.norm(r)) <= 1e-12


def test_enough_iterations_give_the_dense_solve(lvl):
    O, q, qc, l = lvl["O"], lvl["q"], lvl["qc"], lvl["l"]
    N = qc.size
    if N > 1200:
        pytest.skip("dense reference on the small levels only")
    O.pmg_setup(q, [1, 1], 3.0, 1.5, coarse="mbnk", mbnk_maxit=N, mbnk_tol=1e-13)
    A = np.stack([O.mbnk_matvec(np.eye(N)[j].reshape(qc.shape), l).ravel() for j in range(N)], axis=1)
    r = np.random.default_rng(3).standard_normal(qc.shape)
    d, k, rel = O.mbnk_solve(r, l)
    ref = np.linalg.solve(A, r.ravel())
    assert np.linalg.norm(d.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)
    assert rel <= 1e-13 and k < N


def test_stopping_rule(lvl):
    O, q, qc, l = lvl["O"], lvl["q"], lvl["qc"], lvl["l"]
    r = np.random.default_rng(4).standard_normal(qc.shape)
    O.pmg_setup(q, [1, 1], 3.0, 1.5, coarse="mbnk", mbnk_maxit=20, mbnk_tol=0.1)
    d, k, rel = O.mbnk_solve(r, l)
    true = np.linalg.norm(r - O.mbnk_matvec(d, l)) / np.linalg.norm(r)
    assert rel <= 0.1 and abs(true - rel) <= 1e-10
    if k > 1:
        O.pmg_setup(q, [1, 1], 3.0, 1.5, coarse="mbnk", mbnk_maxit=k - 1, mbnk_tol=0.1)
        _, k2, rel2 = O.mbnk_solve(r, l)
        assert k2 == k - 1 and rel2 > 0.1


@pytest.fixture(scope="module")
def small():
    mesh = w.box2d(3, 3, 10, 10, qg=2, warp=0.1)
    ph = w.Physics(mu=0.02, qinf=w.freestream(2, 0.3))
    q = angled_flow(mesh, 2)
    O = oracle.Oracle(mesh, ph, [2])
    N = q.size
    J = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1e-5
        J[:, j] = (O.residual(q + e.reshape(q.shape)) - O.residual(q - e.reshape(q.shape))).ravel() / 2e-5
    return dict(mesh=mesh, ph=ph, q=q, J=J, N=N)


def test_one_level_exact_mbnk_step_is_the_linear_solve(small):
    mesh, ph, q, J, N = small["mesh"], small["ph"], small["q"], small["J"], small["N"]
    O = oracle.Oracle(mesh, ph, [2])
    c = 4.0
    O.pmg_setup(q, [1], c, 0.0, coarse="mbnk", mbnk_maxit=N, mbnk_tol=1e-14)
    X = 1e-3 * np.random.default_rng(5).standard_normal(q.shape)
    Y = O.pmg_apply(q, O.residual(q), X)
    ref = np.linalg.solve(c * np.eye(N) - J, X.ravel())
    assert np.linalg.norm(Y.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)


def test_two_level_cycle_with_mbnk_keeps_the_fixed_point(small):
    mesh, ph, q, J, N = small["mesh"], small["ph"], small["q"], small["J"], small["N"]
    dt = 0.5
    c = 1.0 / dt + 1.0 / (0.4358665215 * dt)
    O = oracle.Oracle(mesh, ph, [2, 1])
    O.pmg_setup(q, [40, 2], c, 0.0, coarse="mbnk")
    X = 1e-3 * np.random.default_rng(6).standard_normal(q.shape) / math.sqrt(N)
    Y = O.pmg_apply(q, O.residual(q), X)
    ref = np.linalg.solve(c * np.eye(N) - J, X.ravel())
    assert np.linalg.norm(Y.ravel() - ref) <= 1e-4 * np.linalg.norm(ref)


def test_esdirk_step_with_mbnk_reaches_the_same_state():
    mesh = w.box2d(4, 4, 10, 10, qg=2, warp=0.1)
    ph = w.Physics(mu=0.01, qinf=w.freestream(2, 0.5))
    X = w.solution_point_coords(mesh, 2)
    q0 = np.ascontiguousarray(w.isentropic_vortex(X, 5, 5, 5.0, 0.5, 10, 10))
    dt = 10.0 * w.explicit_dt(mesh, 2, q0)
    O = oracle.Oracle(mesh, ph, [2, 1])
    A, b, _ = TB.esdirk3()
    out = {}
    for coarse in ("ej", "mbnk"):
        o = O.opts(kdim=30, maxit_gmres=300, max_ptc=40, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-12,
                   dtau=dt, inv_dtau_star=1.0 / dt, coarse=coarse)
        out[coarse] = O.esdirk_step(A, b, dt, q0, o)
    (qe, se), (qm, sm) = out["ej"], out["mbnk"]
    assert se["converged"] and sm["converged"]
    assert np.abs(qm - qe).max() <= 1e-9 * np.abs(qe).max()
