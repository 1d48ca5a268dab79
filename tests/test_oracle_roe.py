"""Pins of the oracle's Roe flux (the original Roe solver the paper runs its unsteady cases
with, Sec. 4.2), checked against what defines it rather than against its own formula:

  - consistency: F(q, q, n) = f(q) . n;
  - conservation: F(qL, qR, n) = -F(qR, qL, -n);
  - Roe's construction: F = (fL + fR) . n / 2 - |A| (qR - qL) / 2, with A the flux Jacobian
    along n at the Roe-averaged state (taken here by central differences of the oracle's
    physical flux, |A| from numpy's eigen-decomposition), and A (qR - qL) = (fR - fL) . n;
  - full upwinding when every wave speed has one sign (supersonic along n): F = f(qL) . n
    or f(qR) . n;
  - exact resolution of a stationary contact and a stationary shear layer: F = (0, p n, 0);
and, at the residual level with the Roe flux: free-stream preservation on a curved O-mesh,
discrete conservation on a periodic mesh, the inviscid order of accuracy on manufactured
solutions and the stability of the operator linearised about a rest state."""
import math

import numpy as np
import pytest

import oracle
from paper_2202_09733_gb300 import workloads as w
import mms

GM1 = w.GAMMA - 1.0


def cons(rho, u, p):
    u = np.asarray(u, dtype=float)
    return np.concatenate([[rho], rho * u, [p / GM1 + 0.5 * rho * u @ u]])


def ctx(d, flux="roe", mu=0.0):
    mesh = w.box2d(2, 2, 1.0, 1.0, qg=1) if d == 2 else w.box3d(2, 1.0)
    return oracle.Oracle(mesh, w.Physics(mu=mu, qinf=np.zeros(d + 2), flux=flux), [1])


def fn(O, q, n):
    return O.inviscid_flux(q).T @ n


def roe_jacobian(O, qL, qR, n):
    """A = d(f . n)/dq at the Roe-averaged state, by central differences of the physical flux."""
    d = O.d
    rL, rR = qL[0], qR[0]
    uL, uR = qL[1:1 + d] / rL, qR[1:1 + d] / rR
    pL = GM1 * (qL[-1] - 0.5 * rL * uL @ uL)
    pR = GM1 * (qR[-1] - 0.5 * rR * uR @ uR)
    HL, HR = (qL[-1] + pL) / rL, (qR[-1] + pR) / rR
    sL, sR = math.sqrt(rL), math.sqrt(rR)
    ut = (sL * uL + sR * uR) / (sL + sR)
    Ht = (sL * HL + sR * HR) / (sL + sR)
    rt = sL * sR
    Et = (Ht + GM1 * 0.5 * ut @ ut) / w.GAMMA        # H = gamma E - (gamma - 1) |u|^2 / 2
    qt = np.concatenate([[rt], rt * ut, [rt * Et]])
    nv = d + 2
    A = np.zeros((nv, nv))
    for j in range(nv):
        h = 1e-6 * max(1.0, abs(qt[j]))
        a, b = qt.copy(), qt.copy()
        a[j] += h
        b[j] -= h
        A[:, j] = (fn(O, a, n) - fn(O, b, n)) / (2 * h)
    return A


def absm(A):
    lam, V = np.linalg.eig(A)
    return ((V * np.abs(lam.real)) @ np.linalg.inv(V)).real


def random_pair(rng, d, mach):
    out = []
    for _ in range(2):
        rho = rng.uniform(0.5, 2.0)
        p = rng.uniform(0.5, 2.0)
        c = math.sqrt(w.GAMMA * p / rho)
        u = rng.standard_normal(d)
        u *= mach * c / np.linalg.norm(u)
        out.append(cons(rho, u, p))
    n = rng.standard_normal(d)
    n *= rng.uniform(0.2, 3.0) / np.linalg.norm(n)    # scaled normal, as on a curved face
    return out[0], out[1], n


@pytest.mark.parametrize("d", [2, 3])
def test_consistency_and_conservation(d):
    O = ctx(d)
    rng = np.random.default_rng(d)
    for _ in range(20):
        qL, qR, n = random_pair(rng, d, rng.uniform(0.0, 2.0))
        F0 = fn(O, qL, n)
        assert np.allclose(O.common_flux(qL, qL, n), F0, rtol=0, atol=1e-14 * np.abs(F0).max())
        F = O.common_flux(qL, qR, n)
        Fs = O.common_flux(qR, qL, -n)
        assert np.allclose(F, -Fs, rtol=0, atol=1e-14 * np.abs(F).max())


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("mach", [0.05, 0.4, 0.9])
def test_matches_roe_matrix_construction(d, mach):
    O = ctx(d)
    rng = np.random.default_rng(int(100 * mach) + d)
    for _ in range(10):
        qL, qR, n = random_pair(rng, d, mach)
        A = roe_jacobian(O, qL, qR, n)
        fL, fR = fn(O, qL, n), fn(O, qR, n)
        scale = np.abs(fL).max() + np.abs(fR).max()
        assert np.abs(A @ (qR - qL) - (fR - fL)).max() <= 1e-8 * scale      # Roe's property
        Fx = 0.5 * (fL + fR) - 0.5 * absm(A) @ (qR - qL)
        assert np.abs(O.common_flux(qL, qR, n) - Fx).max() <= 1e-8 * scale


@pytest.mark.parametrize("d", [2, 3])
def test_supersonic_is_full_upwinding(d):
    O = ctx(d)
    rng = np.random.default_rng(7 + d)
    n = rng.standard_normal(d)
    nh = n / np.linalg.norm(n)
    for sign in (1.0, -1.0):
        for _ in range(5):
            qs = []
            for _ in range(2):
                rho, p = rng.uniform(0.8, 1.2), rng.uniform(0.8, 1.2)
                c = math.sqrt(w.GAMMA * p / rho)
                u = sign * rng.uniform(2.5, 3.0) * c * nh + 0.3 * c * rng.standard_normal(d)
                qs.append(cons(rho, u, p))
            F = O.common_flux(qs[0], qs[1], n)
            up = fn(O, qs[0] if sign > 0 else qs[1], n)
            assert np.abs(F - up).max() <= 1e-13 * np.abs(up).max()
            # Rusanov keeps its dissipation here: the two fluxes differ
            assert np.abs(O.common_flux(qs[0], qs[1], n, kind="rusanov") - up).max() > 1e-6 * np.abs(up).max()


@pytest.mark.parametrize("d", [2, 3])
def test_stationary_contact_and_shear_are_exact(d):
    O = ctx(d)
    n = np.array([0.6, -0.8, 0.0][:d]) * 1.7
    nh = n / np.linalg.norm(n)
    t = np.array([0.8, 0.6, 0.0][:d])                 # tangent to the face
    p = 0.9
    cases = [(cons(1.0, np.zeros(d), p), cons(2.5, np.zeros(d), p)),          # contact
             (cons(1.0, 0.4 * t, p), cons(1.0, -0.3 * t, p))]                 # shear layer
    for qL, qR in cases:
        F = O.common_flux(qL, qR, n)
        exact = np.concatenate([[0.0], p * n, [0.0]])
        assert np.abs(F - exact).max() <= 1e-15
        Fr = O.common_flux(qL, qR, n, kind="rusanov")
        assert np.abs(Fr - exact).max() > 1e-3                               # Rusanov smears it


def test_residual_freestream_omesh():
    mesh = w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3)
    f = mesh["faces"].copy()
    f[f[:, 5] == 2, 5] = 1
    mesh["faces"] = f
    qinf = w.freestream(2, 0.3)
    O = oracle.Oracle(mesh, w.Physics(mu=0.01, qinf=qinf, flux="roe"), [4, 2, 1])
    rho, vel = qinf[0], qinf[1:3] / qinf[0]
    pr = GM1 * (qinf[3] - 0.5 * rho * vel @ vel)
    scale = (qinf[3] + pr) * 2.0 / mesh["h_min"]
    for l, p in enumerate(O.levels):
        R = O.residual(np.broadcast_to(qinf[:, None, None], O.shape(l)).copy(), l)
        assert np.abs(R).max() <= 1e-14 * scale * (p + 1) ** 2


@pytest.mark.parametrize("p", [2, 3])
def test_residual_conservation_periodic(p):
    mesh = w.box2d(5, 4, 10, 8, qg=2, warp=0.15)
    O = oracle.Oracle(mesh, w.Physics(mu=0.05, qinf=w.freestream(2, 0.5), flux="roe"), [p])
    X = w.solution_point_coords(mesh, p)
    R = O.residual(w.isentropic_vortex(X, 5, 4, 5.0, 0.5, 10, 8))
    J = O.jacobian_det()
    t = oracle.table(p)
    Wt = np.outer(t["w"], t["w"]).ravel()
    tot = np.einsum("i,ie,vie->v", Wt, J, R)
    scale = np.einsum("i,ie,vie->v", Wt, J, np.abs(R))
    assert np.all(np.abs(tot) <= 1e-13 * scale)


@pytest.mark.parametrize("p", [2, 3])
def test_residual_order_inviscid(p):
    s0, t0 = mms.exact_rhs(2, 0.0)
    errs = []
    for n in (4, 8, 16):
        mesh = w.box2d(n, n, 2 * math.pi, 2 * math.pi, qg=2, warp=0.1)
        X = w.solution_point_coords(mesh, p)
        R = oracle.Oracle(mesh, w.Physics(mu=0.0, qinf=np.zeros(4), flux="roe"), [p]).residual(s0(X))
        errs.append(np.sqrt(np.mean((R - t0(X)) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] >= p - 0.2


def test_residual_linearised_stable():
    mesh = w.box2d(3, 3, 3.0, 3.0, qg=2, warp=0.1)
    qinf = w.freestream(2, 0.3)
    qinf[1] = 0.0
    qinf[3] = (1 / (1.4 * 0.09)) / 0.4
    O = oracle.Oracle(mesh, w.Physics(mu=0.2, qinf=qinf, flux="roe"), [2])
    q = np.broadcast_to(qinf[:, None, None], O.shape(0)).copy()
    q[1] += 1e-3                       # a slow drift, so the entropy wave speed is not zero
    R0 = O.residual(q).ravel()
    N = q.size
    J = np.zeros((N, N))
    for j in range(N):
        qq = q.ravel().copy()
        qq[j] += 1e-6
        J[:, j] = (O.residual(qq.reshape(q.shape)).ravel() - R0) / 1e-6
    ev = np.linalg.eigvals(J)
    assert ev.real.max() <= 1e-7 * np.abs(ev).max()
