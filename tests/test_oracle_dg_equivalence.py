"""FR with DG-recovering correction functions on Gauss-Legendre points is nodal DG
(Huynh's equivalence; Sec. 2.1 names FR without fixing its correction functions, and the
oracle reads them as the DG ones).  Pin: on affine periodic quads with mu = 0 the
oracle's R(q) equals a textbook weak-form nodal DG residual written here independently,

    w_a w_b J dq_ab/dt = sum_c w_c w_b J (d phi_ab/dx)(c, b) f_x(q_cb) + (same in y)
                         - sum over faces of (h/2) w phi_ab(face point) f*.n_out,

with numpy's Gauss-Legendre rule, Lagrange derivatives from numpy polynomials, traces
interpolated from the nodes, element neighbours found from element centres, and the
Rusanov flux along the unit outward normal.  The two agree to rounding for p = 1..4 on
random smooth states (the weak form integrates by parts exactly under the 2p+1-exact
rule)."""
import numpy as np
import pytest

import oracle
from paper_2202_09733_gb300 import workloads as w

G = 1.4


def lagrange_tables(p):
    x, wq = np.polynomial.legendre.leggauss(p + 1)
    n = p + 1
    D = np.zeros((n, n))          # D[c, a] = l_a'(x_c)
    lm, lp = np.zeros(n), np.zeros(n)
    for a in range(n):
        others = np.delete(x, a)
        poly = np.poly1d(others, r=True) / np.prod(x[a] - others)
        D[:, a] = poly.deriv()(x)
        lm[a], lp[a] = poly(-1.0), poly(1.0)
    return x, wq, D, lm, lp


def euler_flux(q, k):
    rho, mx, my, E = q
    u, v = mx / rho, my / rho
    p = (G - 1.0) * (E - 0.5 * (mx * u + my * v))
    un = u if k == 0 else v
    return np.stack([rho * un, mx * un + (p if k == 0 else 0.0), my * un + (p if k == 1 else 0.0), (E + p) * un])


def rusanov(qL, qR, k):
    """numerical flux along +axis k between a left state and a right state"""
    def lam(q):
        rho = q[0]
        u = q[1 + k] / rho
        p = (G - 1.0) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / rho)
        return np.abs(u) + np.sqrt(G * p / rho)
    lm = np.maximum(lam(qL), lam(qR))
    return 0.5 * (euler_flux(qL, k) + euler_flux(qR, k)) - 0.5 * lm * (qR - qL)


def dg_residual(q, mesh, p):
    nx, ny = mesh["shape"]
    Lx, Ly = mesh["L"]
    hx, hy = Lx / nx, Ly / ny
    n = p + 1
    x, wq, D, lm, lp = lagrange_tables(p)
    X = w.solution_point_coords(mesh, p)
    E = q.shape[2]
    # element grid position from the centre; point ordering checked from the coordinates
    xc, yc = X[0].mean(axis=0), X[1].mean(axis=0)
    ix = np.rint(xc / hx - 0.5).astype(int)
    iy = np.rint(yc / hy - 0.5).astype(int)
    at = {(i, j): e for e, (i, j) in enumerate(zip(ix, iy))}
    Xg = X.reshape(2, n, n, E)                  # [c][i1][i0][e]
    assert np.allclose(Xg[0][0, :, 0], (ix[0] + 0.5 * (x + 1)) * hx)
    assert np.allclose(Xg[1][:, 0, 0], (iy[0] + 0.5 * (x + 1)) * hy)
    Q = q.reshape(4, n, n, E)                   # [v][i1 (y)][i0 (x)][e]
    J = hx * hy / 4.0
    R = np.zeros_like(Q)
    fx, fy = euler_flux(Q, 0), euler_flux(Q, 1)
    # volume: sum_c w_c l_a'(x_c) f(c) * (J * 2/h) * w_b
    R += np.einsum("c,ca,vbce,b->vbae", wq, D, fx, wq) * (J * 2.0 / hx)
    R += np.einsum("c,cb,vcae,a->vbae", wq, D, fy, wq) * (J * 2.0 / hy)
    # traces
    qxm = np.einsum("a,vbae->vbe", lm, Q)       # at xi0 = -1, per row b
    qxp = np.einsum("a,vbae->vbe", lp, Q)
    qym = np.einsum("b,vbae->vae", lm, Q)
    qyp = np.einsum("b,vbae->vae", lp, Q)
    right = np.array([at[((i + 1) % nx, j)] for i, j in zip(ix, iy)])
    up = np.array([at[(i, (j + 1) % ny)] for i, j in zip(ix, iy)])
    Fx = rusanov(qxp, qxm[:, :, right], 0)     # on the +x face of every element, along +x
    Fy = rusanov(qyp, qym[:, :, up], 1)
    left = np.empty(E, dtype=int)
    left[right] = np.arange(E)
    down = np.empty(E, dtype=int)
    down[up] = np.arange(E)
    # - (h/2) w phi(face) f*.n_out on the four faces
    R -= np.einsum("a,vbe,b->vbae", lp, Fx, wq) * (hy / 2.0)
    R += np.einsum("a,vbe,b->vbae", lm, Fx[:, :, left], wq) * (hy / 2.0)
    R -= np.einsum("b,vae,a->vbae", lp, Fy, wq) * (hx / 2.0)
    R += np.einsum("b,vae,a->vbae", lm, Fy[:, :, down], wq) * (hx / 2.0)
    R /= (np.outer(wq, wq) * J)[None, :, :, None]
    return R.reshape(q.shape)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fr_residual_is_nodal_dg(p):
    mesh = w.box2d(5, 4, 10.0, 6.0, qg=2, warp=0.0)
    O = oracle.Oracle(mesh, w.Physics(mu=0.0, qinf=np.zeros(4)), [p])
    X = w.solution_point_coords(mesh, p)
    rng = np.random.default_rng(p)
    k = rng.uniform(0.5, 1.5, size=(4, 2))
    s = [np.sin(k[i, 0] * X[0] + k[i, 1] * X[1] + i) for i in range(4)]
    q = np.ascontiguousarray(w.prim_to_cons(1.0 + 0.1 * s[0], [0.6 + 0.2 * s[1], -0.3 + 0.2 * s[2]],
                                            (1.0 / (1.4 * 0.25)) * (1.0 + 0.1 * s[3])))
    R_or = O.residual(q)
    R_dg = dg_residual(q, mesh, p)
    assert np.abs(R_or - R_dg).max() <= 1e-12 * np.abs(R_dg).max()
