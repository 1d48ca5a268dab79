"""Pins of the oracle's solver layer.

  Jv (Eq. 8)         forward-difference error is O(eps) against a central difference
  element blocks     equal, bit for bit, to the diagonal blocks of the full-residual FD
                     Jacobian (brute force, column by column)
  LU                 block solves equal numpy's dense solves
  pMG (Sec. 3.2)     one fine-level pseudo step with 1/dtau* = 0 is the element-Jacobi
                     preconditioner diag(A)^{-1} X (the special case the paper notes);
                     a two-level cycle whose coarse level has the same degree equals the
                     one-level smoother with 2 n0 + n1 steps; many smoothing steps reach
                     the fixed point A^{-1} X of the preconditioner's pseudo-time system
  FGMRES             converges to the dense direct solve of the FD Jacobian system
  ESDIRK3 / ROS34PW2 order conditions, L-stability, observed order 3 on the NS system
  steady PTC + SER   converges by 7 orders on a small stretched cylinder mesh
  pMG solver         one iteration with one level and one smoothing step is the
                     element-Jacobi pseudo step q + diag(A)^{-1} R(q); the two-level
                     solver reduces the residual by three orders in 150 iterations
"""
import math

import numpy as np
import pytest

import oracle
from oracle import tableaux as TB
from paper_2202_09733_gb300 import workloads as w
from smooth_state import angled_flow


@pytest.fixture(scope="module")
def small():
    mesh = w.box2d(3, 3, 10, 10, qg=2, warp=0.1)
    ph = w.Physics(mu=0.02, qinf=w.freestream(2, 0.3))
    O = oracle.Oracle(mesh, ph, [2, 1])
    q = angled_flow(mesh, 2)
    Rq = O.residual(q)
    N = q.size
    Jd = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1e-5
        Jd[:, j] = (O.residual(q + e.reshape(q.shape)) - O.residual(q - e.reshape(q.shape))).ravel() / 2e-5
    return dict(mesh=mesh, ph=ph, O=O, q=q, Rq=Rq, J=Jd, N=N)


def test_jvp_first_order_in_eps(small):
    O, q, Rq = small["O"], small["q"], small["Rq"]
    v = np.random.default_rng(1).standard_normal(q.shape)
    v /= np.linalg.norm(v)
    ref = -(small["J"] @ v.ravel())
    errs = [np.linalg.norm(O.jvp(q, Rq, v, eps, 0.0).ravel() - ref) / np.linalg.norm(ref)
            for eps in (1e-3, 1e-4, 1e-5)]
    assert 8.0 < errs[0] / errs[1] < 12.0 and 8.0 < errs[1] / errs[2] < 12.0
    # shift term enters linearly
    a1 = O.jvp(q, Rq, v, 1e-6, 0.0)
    a2 = O.jvp(q, Rq, v, 1e-6, 3.0)
    assert np.allclose(a2 - a1, 3.0 * v, rtol=0, atol=1e-14)


def test_element_blocks_equal_full_jacobian_blocks(small):
    O, q, Rq = small["O"], small["q"], small["Rq"]
    nd = q.shape[0] * q.shape[1]
    for e0 in (0, 4, 8):
        cols = []
        for j in range(nd):
            qq = q.copy().reshape(nd, -1)
            eps = 1e-7 * max(1.0, abs(qq[j, e0]))
            qq[j, e0] = qq[j, e0] + eps
            cols.append((O.residual(qq.reshape(q.shape)) - Rq).reshape(nd, -1)[:, e0] / eps)
        Mfull = 2.5 * np.eye(nd) - np.stack(cols, axis=1)
        Mb = O.elem_blocks(q, 2.5, [e0])[0]
        off = ~np.eye(nd, dtype=bool)
        assert np.array_equal(Mb[off], Mfull[off])
        assert np.allclose(np.diag(Mb), np.diag(Mfull), rtol=1e-15, atol=0)


def test_block_solve_equals_dense_solve(small):
    O, q = small["O"], small["q"]
    c = 3.0
    O.pmg_setup(q, [1], c, 0.0)
    M = O.elem_blocks(q, c, np.arange(small["mesh"]["E"]))
    x = np.random.default_rng(2).standard_normal(q.shape)
    y = O.block_solve(x)
    nd = M.shape[1]
    ref = np.stack([np.linalg.solve(M[e], x.reshape(nd, -1)[:, e]) for e in range(M.shape[0])], axis=1)
    assert np.allclose(y.reshape(nd, -1), ref, rtol=1e-12, atol=1e-14)


def test_pmg_one_step_is_element_jacobi(small):
    O, q, Rq = small["O"], small["q"], small["Rq"]
    c = 1.0 / 0.5 + 1.0 / (0.4358665215 * 0.5)
    O.pmg_setup(q, [1], c, 0.0)
    X = np.random.default_rng(3).standard_normal(q.shape)
    Y = O.pmg_apply(q, Rq, X)
    M = O.elem_blocks(q, c, np.arange(small["mesh"]["E"]))
    nd = M.shape[1]
    ref = np.stack([np.linalg.solve(M[e], X.reshape(nd, -1)[:, e]) for e in range(M.shape[0])], axis=1)
    assert np.abs(Y.reshape(nd, -1) - ref).max() <= 1e-13 * np.abs(q).max()


def test_pmg_same_degree_coarse_level_is_extra_smoothing(small):
    mesh, ph, q, Rq = small["mesh"], small["ph"], small["q"], small["Rq"]
    X = np.random.default_rng(4).standard_normal(q.shape)
    c, ids = 5.0, 2.0
    O2 = oracle.Oracle(mesh, ph, [2, 2])
    O2.pmg_setup(q, [1, 1], c, ids)
    Ya = O2.pmg_apply(q, Rq, X)
    O1 = oracle.Oracle(mesh, ph, [2])
    O1.pmg_setup(q, [3], c, ids)
    Yb = O1.pmg_apply(q, Rq, X)
    assert np.abs(Ya - Yb).max() <= 1e-12 * np.abs(Yb).max()


@pytest.mark.parametrize("levels,nsmooth", [([2], [80]), ([2, 1], [40, 40])])
def test_pmg_fixed_point_is_linear_solve(small, levels, nsmooth):
    mesh, ph, q, Rq, J, N = small["mesh"], small["ph"], small["q"], small["Rq"], small["J"], small["N"]
    dt = 0.5
    c = 1.0 / dt + 1.0 / (0.4358665215 * dt)
    O = oracle.Oracle(mesh, ph, levels)
    O.pmg_setup(q, nsmooth, c, 0.0)
    X = 1e-3 * np.random.default_rng(5).standard_normal(q.shape) / math.sqrt(N)
    Y = O.pmg_apply(q, Rq, X)
    ref = np.linalg.solve(c * np.eye(N) - J, X.ravel())
    assert np.linalg.norm(Y.ravel() - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("use_pmg", [False, True])
def test_fgmres_matches_dense_solve(small, use_pmg):
    O, q, Rq, J, N = small["O"], small["q"], small["Rq"], small["J"], small["N"]
    dt = 0.5
    c = 1.0 / dt + 1.0 / (0.4358665215 * dt)
    b = np.random.default_rng(6).standard_normal(q.shape)
    ref = np.linalg.solve(c * np.eye(N) - J, b.ravel())
    if use_pmg:
        O.pmg_setup(q, [2, 2], c, 1.0 / dt)
    x, st = O.gmres(q, Rq, b, kdim=N, tol=1e-9, maxit=N, shift=c, use_pmg=use_pmg)
    assert np.linalg.norm(x.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)
    assert st["relres"] <= 1e-6


def test_tableaux_order_conditions():
    A, b, c = TB.esdirk3()
    assert abs(b.sum() - 1) < 1e-15 and abs(b @ c - 0.5) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15 and abs(b @ A @ c - 1 / 6) < 1e-15
    # L-stability of a stiffly accurate ESDIRK: R(z) -> 0 as z -> -inf
    z = -1e8
    R = 1 + z * b @ np.linalg.solve(np.eye(4) - z * A, np.ones(4))
    assert abs(R) < 1e-6
    gam, alpha, G, bb = TB.ros34pw2_standard()
    beta = alpha + G - np.diag(np.diag(G))
    bp, al = beta.sum(1), alpha.sum(1)
    assert abs(bb.sum() - 1) < 1e-15 and abs(bb @ bp - (0.5 - gam)) < 1e-15
    assert abs(bb @ al ** 2 - 1 / 3) < 1e-15 and abs(bb @ (beta @ bp) - (1 / 6 - gam + gam * gam)) < 1e-15
    # stiff accuracy: b is the last row of alpha + Gamma
    assert np.allclose(bb, (alpha + G)[3], atol=1e-15)
    # transformed coefficients reproduce the scalar linear test equation
    g, a, cc, m = TB.ros34pw2()
    lam, h = -0.7, 0.3
    Y = []
    for i in range(4):
        rhs = lam * (1 + sum(a[i, j] * Y[j] for j in range(i))) + sum(cc[i, j] * Y[j] for j in range(i)) / h
        Y.append(rhs / (1 / (g * h) - lam))
    y1 = 1 + sum(m[j] * Y[j] for j in range(4))
    # the same step in the standard form
    K = []
    for i in range(4):
        s = lam * h * (1 + sum(alpha[i, j] * K[j] for j in range(i))) + lam * h * sum(G[i, j] * K[j] for j in range(i))
        K.append(s / (1 - lam * h * gam))
    assert abs(y1 - (1 + bb @ np.array(K))) < 1e-14


def _stability(A, b, z):
    s = len(b)
    return 1 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


@pytest.mark.parametrize("name,order", [("esdirk2", 2), ("esdirk4", 4)])
def test_paper_esdirk_tableaux(name, order):
    """The paper's ESDIRK2 / ESDIRK4: every order condition up to the scheme's order
    (and the first third-order one fails for ESDIRK2), stage order 2 (explicit first stage,
    a_i1 = ... sums to c_i with sum_j a_ij c_j = c_i^2 / 2), stiff accuracy, L-stability
    (R(-inf) = 0) and A-stability (|R| <= 1 on the imaginary axis and in the left half plane)."""
    A, b, c = getattr(TB, name)()
    s = len(b)
    assert np.all(A[0] == 0) and np.all(np.triu(A, 1) == 0) and np.allclose(np.diag(A)[1:], A[1, 1])
    assert np.array_equal(b, A[-1])
    assert np.allclose(A.sum(1), c, atol=1e-15)
    conds = [(b.sum(), 1.0), (b @ c, 0.5)]
    third = [(b @ c ** 2, 1 / 3), (b @ A @ c, 1 / 6)]
    fourth = [(b @ c ** 3, 1 / 4), (b @ (c * (A @ c)), 1 / 8), (b @ A @ c ** 2, 1 / 12), (b @ A @ A @ c, 1 / 24)]
    if order >= 3:
        conds += third
    if order >= 4:
        conds += fourth
    for got, want in conds:
        assert abs(got - want) < 2e-15, (got, want)
    if order == 2:
        assert abs(third[0][0] - 1 / 3) > 1e-3
    assert np.allclose((A @ c)[1:], c[1:] ** 2 / 2, atol=2e-15)
    assert abs(_stability(A, b, -1e8)) < 1e-6
    for y in np.logspace(-3, 4, 200):
        assert abs(_stability(A, b, 1j * y)) <= 1 + 1e-12
    rng = np.random.default_rng(order)
    for z in -np.abs(rng.standard_normal(200)) * 10 + 1j * rng.standard_normal(200) * 10:
        assert abs(_stability(A, b, z)) <= 1 + 1e-12


def _march(O, kind, q0, T, dt):
    q = q0.copy()
    for _ in range(int(round(T / dt))):
        if kind.startswith("esdirk"):
            A, b, _ = getattr(TB, kind)()
            opts = O.opts(kdim=40, maxit_gmres=200, max_ptc=30, nsmooth=(2, 2), tol_gmres=1e-3,
                          tol_newton=1e-10, dtau=dt, inv_dtau_star=1.0 / dt)
            q, st = O.esdirk_step(A, b, dt, q, opts)
            assert st["converged"]
        else:
            g, a, c, m = TB.ros34pw2()
            opts = O.opts(kdim=40, maxit_gmres=200, nsmooth=(2, 2), tol_gmres=1e-7, inv_dtau_star=1.0 / dt)
            q, st = O.row_step(g, a, c, m, dt, q, opts)
    return q


@pytest.mark.parametrize("kind,min_rate", [("esdirk2", 1.8), ("esdirk3", 2.6), ("esdirk4", 3.7), ("row", 2.6)])
def test_observed_temporal_order(kind, min_rate):
    mesh = w.box2d(2, 2, 10, 10, qg=2, warp=0.1)
    O = oracle.Oracle(mesh, w.Physics(mu=0.02, qinf=w.freestream(2, 0.3)), [2, 1])
    q0 = angled_flow(mesh, 2, amp=0.1)
    T = 0.4
    ref = _march(O, kind, q0, T, 0.0125)
    errs = np.array([np.abs(_march(O, kind, q0, T, dt) - ref).max() for dt in (0.2, 0.1)])
    rate = math.log2(errs[0] / errs[1])
    assert rate > min_rate


def test_steady_ptc_ser_converges():
    W = w.cylinder_steady(nr=6, nt=12, p=2, levels=[2, 1], mach=0.2, re=40)
    O = oracle.Oracle(W.mesh, W.phys, W.levels)
    opts = O.opts(kdim=30, maxit_gmres=60, nsmooth=(2, 2), tol_gmres=1e-3, inv_dtau_star=-1.0)
    dtau0 = 0.1 * W.mesh["h_min"] / (1.0 + 1.0 / 0.2)
    q, st = O.ptc_steady(W.q0, dtau0, 1e6, 1e-7, 80, opts)
    assert st["converged"] and st["final_res"] <= 1e-7


def test_library_tableaux_match_oracle_tableaux():
    from paper_2202_09733_gb300 import tableaux as GT
    for name in ("esdirk2", "esdirk3", "esdirk4"):
        A1, b1, _ = getattr(TB, name)()
        A2, b2 = getattr(GT, name)()
        assert np.array_equal(A1, A2) and np.array_equal(b1, b2), name
    for x, y in zip(TB.ros34pw2(), GT.ros34pw2()):
        assert np.allclose(x, y, rtol=1e-15, atol=1e-15)


def test_pmg_solver_one_level_step_is_element_jacobi():
    W = w.cylinder_steady(nr=6, nt=12, p=2, levels=[2, 1], mach=0.2, re=40)
    O = oracle.Oracle(W.mesh, W.phys, W.levels)
    dtau = 0.1 * W.mesh["h_min"] / (1.0 + 1.0 / 0.2)
    opts = O.opts(nsmooth=(1,), inv_dtau_star=0.0)
    q1, st = O.pmg_steady(W.q0, dtau, dtau, 0.0, 1, opts)
    assert st["n_ptc"] == 1
    R0 = O.residual(W.q0)
    O.pmg_setup(W.q0, [1], 1.0 / dtau, 0.0)      # blocks (1/dtau) I - J_ee at q0
    assert np.array_equal(q1, W.q0 + O.block_solve(R0))


def test_pmg_solver_reduces_the_residual():
    """The nonlinear solver converges linearly (the paper's reason to prefer JFNK-pMG):
    more than three orders in 150 iterations with SER on the small cylinder mesh, with no
    growth over its last iterations."""
    W = w.cylinder_steady(nr=6, nt=12, p=2, levels=[2, 1], mach=0.2, re=40)
    O = oracle.Oracle(W.mesh, W.phys, W.levels)
    dtau0 = 0.1 * W.mesh["h_min"] / (1.0 + 1.0 / 0.2)
    q, st = O.pmg_steady(W.q0, dtau0, 1e6, 0.0, 150, O.opts(nsmooth=(2, 2), inv_dtau_star=-1.0))
    h = st["hist"]
    assert st["n_ptc"] == 150 and h[-1] < 1e-3 * h[0]
    assert np.all(h[-30:] <= 1.05 * h[-31:-1])


def test_pmg_nonlinear_stage_solver_one_update_is_element_jacobi():
    """ESDIRK3 with the pMG nonlinear stage solver, one level, one smoothing step, 1/dtau* = 0
    and one update per stage (max_ptc = 1): every stage does q <- q^n - M^-1 F(q^n) with
    M = (1/dtau + 1/(a_ii dt)) I - dR_e/dq_e at q^n, and the step is q^n + dt sum_j b_j R(Q_j);
    rebuilt here in numpy from the residual and the element blocks."""
    mesh = w.box2d(3, 3, 10, 10, qg=2, warp=0.1)
    ph = w.Physics(mu=0.02, qinf=w.freestream(2, 0.3))
    O = oracle.Oracle(mesh, ph, [2])
    qn = angled_flow(mesh, 2)
    A, b, _ = TB.esdirk3()
    dt, dtau = 0.4, 0.7
    o = O.opts(nsmooth=(1,), max_ptc=1, tol_newton=0.0, dtau=dtau, inv_dtau_star=0.0, nonlinear="pmg")
    q_or, st = O.esdirk_step(A, b, dt, qn, o)
    s = len(b)
    c = 1.0 / dtau + 1.0 / (A[1, 1] * dt)
    E = mesh["E"]
    M = O.elem_blocks(qn, c, np.arange(E))
    nd = M.shape[1]
    Rs = [O.residual(qn)]
    for i in range(1, s):
        adt = A[i, i] * dt
        sv = qn + dt * sum(A[i, j] * Rs[j] for j in range(i))
        F = (qn - sv) / adt - O.residual(qn)
        dq = np.stack([np.linalg.solve(M[e], -F.reshape(nd, E)[:, e]) for e in range(E)], axis=1).reshape(qn.shape)
        Rs.append(O.residual(qn + dq))
    ref = qn + dt * sum(b[j] * Rs[j] for j in range(s))
    assert st["n_ptc"] == s - 1 and st["n_gmres"] == 0
    assert np.abs(q_or - ref).max() <= 1e-12 * np.abs(ref).max()


def test_pmg_nonlinear_stage_solver_reaches_the_jfnk_state():
    mesh = w.box2d(4, 4, 10, 10, qg=2, warp=0.1)
    ph = w.Physics(mu=0.01, qinf=w.freestream(2, 0.5))
    X = w.solution_point_coords(mesh, 2)
    q0 = np.ascontiguousarray(w.isentropic_vortex(X, 5, 5, 5.0, 0.5, 10, 10))
    dt = 10.0 * w.explicit_dt(mesh, 2, q0)
    O = oracle.Oracle(mesh, ph, [2, 1])
    A, b, _ = TB.esdirk3()
    out = {}
    for nl in ("jfnk", "pmg"):
        o = O.opts(kdim=30, maxit_gmres=300, max_ptc=400, nsmooth=(2, 2), tol_gmres=1e-2, tol_newton=1e-11,
                   dtau=dt, inv_dtau_star=1.0 / dt, nonlinear=nl)
        out[nl] = O.esdirk_step(A, b, dt, q0, o)
    (qj, sj), (qp, sp) = out["jfnk"], out["pmg"]
    assert sj["converged"] and sp["converged"] and sp["n_gmres"] == 0
    assert sp["n_ptc"] > sj["n_ptc"]            # V-cycles converge linearly, Newton faster
    assert np.abs(qp - qj).max() <= 1e-9 * np.abs(qj).max()
