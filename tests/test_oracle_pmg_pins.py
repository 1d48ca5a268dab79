"""Pins of the oracle's tensor-product p-transfers and of its multi-level coarse correction
(Eqs. 13-18; Eqs. 22-26).

Transfers (Eqs. 17-18), in 2-D and 3-D, against numpy's Gauss rule and polynomials:
  - the restriction of a random nodal field is its L2 projection: the difference
    q - Pi Gamma q is orthogonal to every tensor polynomial of degree <= p1 (checked by an
    independent 12-point-per-direction Gauss-Legendre rule and Lagrange evaluation);
  - the prolongation reproduces tensor polynomials of degree <= p1 exactly;
  - restriction after prolongation is the identity on the coarse space.

Coarse correction (Eqs. 13-16, one V-cycle of the preconditioner, Eqs. 22-26): the
oracle's cycle, with many block-Jacobi pseudo steps on the coarsest level (which then
reaches the coarse fixed point), equals a full-approximation two-grid (or three-grid)
iteration written here directly from the equations:
    pre-smooth:  qh <- qh + M^{-1} (d - (c (qh - b) - (R(qh) - R(b))))
    defect:      r = d - (c (qh - b) - (R(qh) - R(b)))
    coarse:      b1 = Gamma qh,  d1 = Gamma r,   solve  c (y - b1) - (R1(y) - R1(b1)) = d1
                 (Newton with a dense central-difference Jacobian, to round-off)
    correct:     qh <- qh + Pi (y - b1);   post-smooth as before.
Gamma and Pi are applied as Kronecker products of the 1-D operators (not the oracle's
direction-by-direction passes), the element blocks are solved by numpy.linalg.solve and
the coarse problem by Newton, so the cycle's recursion, forcing, signs and transfers are
checked against an independent evaluation.  The same comparison on four plausible
mistakes (coarse forcing dropped, the level's base state restricted instead of qh, defect
sign flipped, y prolonged instead of y - b1) fails by orders of magnitude, so the pin
resolves them.  In the small-input limit the cycle is the
textbook linear two-grid iteration with exact coarse solve, checked against dense
central-difference Jacobians.
"""
import math

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

import oracle
from paper_2202_09733_gb300 import workloads as w
from smooth_state import angled_flow


# ----------------------------------------------------------------- helpers
def _lagrange_matrix(nodes, y):
    """L[a, i] = l_i(y_a) for the Lagrange basis on `nodes`."""
    L = np.ones((len(y), len(nodes)))
    for i in range(len(nodes)):
        for k in range(len(nodes)):
            if k != i:
                L[:, i] *= (y - nodes[k]) / (nodes[i] - nodes[k])
    return L


def _kron_d(A, d):
    K = A
    for _ in range(d - 1):
        K = np.kron(A, K)
    return K


def _apply(K, x):
    """Apply a per-element operator K[out_pt, in_pt] to a [nv][np][E] field."""
    return np.einsum("ij,vje->vie", K, x)


def _mesh(d):
    return w.box2d(2, 2, 10.0, 10.0, qg=2, warp=0.1) if d == 2 else w.box3d(2, 2.0)


TRANSFER_CASES = [(2, 2, 1), (2, 3, 2), (2, 4, 3), (2, 4, 2), (2, 3, 1), (3, 3, 2), (3, 2, 1)]


@pytest.mark.parametrize("d,p0,p1", TRANSFER_CASES)
def test_tensor_restriction_is_l2_projection(d, p0, p1):
    mesh = _mesh(d)
    O = oracle.Oracle(mesh, w.Physics(mu=0.01, qinf=w.freestream(d, 0.3)), [p0, p1])
    x0 = np.random.default_rng(10 * p0 + p1 + d).standard_normal(O.shape(0))
    x1 = O.restrict(x0, 0)
    xq, wq = npleg.leggauss(12)
    n0, n1 = npleg.leggauss(p0 + 1)[0], npleg.leggauss(p1 + 1)[0]
    E0, E1 = _kron_d(_lagrange_matrix(n0, xq), d), _kron_d(_lagrange_matrix(n1, xq), d)
    Wq = _kron_d(np.diag(wq), d).diagonal()
    diff = _apply(E0, x0) - _apply(E1, x1)              # q - Pi Gamma q at the fine quadrature
    # test functions: tensor monomials of degree <= p1 in each direction
    for a in range(p1 + 1):
        for b in range(p1 + 1):
            for c in range(p1 + 1 if d == 3 else 1):
                mono = [xq ** a, xq ** b] + ([xq ** c] if d == 3 else [])
                # slowest index first in the Kronecker product: last direction leftmost
                f = mono[0]
                for m in mono[1:]:
                    f = np.kron(m, f)
                ip = np.einsum("a,a,vae->ve", Wq, f, diff)
                assert np.abs(ip).max() <= 1e-13 * max(1.0, np.abs(x0).max()), (a, b, c)
    # and the projection is not trivial: q itself is not in the coarse space
    assert np.abs(diff).max() > 1e-2


@pytest.mark.parametrize("d,p0,p1", TRANSFER_CASES)
def test_tensor_prolongation_reproduces_coarse_polynomials(d, p0, p1):
    mesh = _mesh(d)
    O = oracle.Oracle(mesh, w.Physics(mu=0.01, qinf=w.freestream(d, 0.3)), [p0, p1])
    n0, n1 = npleg.leggauss(p0 + 1)[0], npleg.leggauss(p1 + 1)[0]

    def nodal(nodes, degs):
        cols = [nodes ** k for k in degs]
        f = cols[0]
        for c in cols[1:]:
            f = np.kron(c, f)
        return f
    rng = np.random.default_rng(d * 100 + p0 * 10 + p1)
    x1 = np.zeros(O.shape(1))
    ref = np.zeros(O.shape(0))
    E, nv = x1.shape[2], x1.shape[0]
    for v in range(nv):
        for e in range(E):
            degs = list(rng.integers(0, p1 + 1, size=d))
            amp = rng.uniform(0.5, 2.0)
            x1[v, :, e] = amp * nodal(n1, degs)
            ref[v, :, e] = amp * nodal(n0, degs)
    x0 = O.prolong(x1, 0)
    assert np.abs(x0 - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("d,p0,p1", TRANSFER_CASES)
def test_restriction_after_prolongation_is_identity(d, p0, p1):
    mesh = _mesh(d)
    O = oracle.Oracle(mesh, w.Physics(mu=0.01, qinf=w.freestream(d, 0.3)), [p0, p1])
    x1 = np.random.default_rng(7).standard_normal(O.shape(1))
    assert np.abs(O.restrict(O.prolong(x1, 0), 0) - x1).max() <= 1e-14 * np.abs(x1).max()


# ------------------------------------------------------- coarse correction (FAS cycle)
def _dense_jacobian(O, l, y, h=1e-6):
    """Central-difference Jacobian dR_l/dq at y (dense, [N, N] over the flattened state)."""
    N = y.size
    J = np.zeros((N, N))
    yf = y.ravel()
    for j in range(N):
        hj = h * max(1.0, abs(yf[j]))
        e = np.zeros(N)
        e[j] = hj
        J[:, j] = (O.residual((yf + e).reshape(y.shape), l) - O.residual((yf - e).reshape(y.shape), l)).ravel() / (2 * hj)
    return J


class FasReference:
    """The multi-level full-approximation cycle of Eqs. 13-16 with the pseudo-time smoother
    of Eq. 26, evaluated with numpy: Kronecker-product transfers, dense element-block
    solves, and an exact (Newton) solve of the coarsest level's equation."""

    def __init__(self, O, levels, q, nsmooth, c, ids):
        self.O, self.levels, self.nsmooth, self.c = O, levels, nsmooth, c
        d = O.d
        self.Gam, self.Pi = [], []
        for l in range(len(levels) - 1):
            G1, P1 = oracle.transfer(levels[l], levels[l + 1])
            self.Gam.append(_kron_d(G1, d))
            self.Pi.append(_kron_d(P1, d))
        # element blocks at the states the preconditioner's set-up uses (the oracle's
        # restriction of q, pinned above)
        self.M = []
        ql = q
        for l in range(len(levels)):
            if l > 0:
                ql = O.restrict(ql, l - 1)
            self.M.append(O.elem_blocks(ql, ids + c, np.arange(O.E), l))

    def block_solve(self, l, x):
        nd = x.shape[0] * x.shape[1]
        xs = x.reshape(nd, -1)
        return np.stack([np.linalg.solve(self.M[l][e], xs[:, e]) for e in range(xs.shape[1])],
                        axis=1).reshape(x.shape)

    def defect(self, l, b, Rb, d, qh):
        return d - (self.c * (qh - b) - (self.O.residual(qh, l) - Rb))

    def coarse_solve(self, l, b, Rb, d, forcing=True):
        """Newton on c (y - b) - (R_l(y) - R_l(b)) = d (with forcing = False, on the equation
        a cycle without the coarse forcing term would solve, c y - R_l(y) = d)."""
        y = b.copy()
        for _ in range(8):
            if forcing:
                F = self.c * (y - b) - (self.O.residual(y, l) - Rb) - d
            else:
                F = self.c * y - self.O.residual(y, l) - d
            A = self.c * np.eye(y.size) - _dense_jacobian(self.O, l, y)
            dy = np.linalg.solve(A, F.ravel()).reshape(y.shape)
            y = y - dy
            if not np.all(np.isfinite(y)) or np.abs(dy).max() <= 1e-15 * np.abs(y - b).max():
                break
        return y

    def cycle(self, l, b, d, mistake=None):
        """qh after one cycle on level l from qh = b with right-hand side d; `mistake` plants
        one error in the coarse correction (for the resolution check only)."""
        Rb = self.O.residual(b, l)
        if l == len(self.levels) - 1:
            return self.coarse_solve(l, b, Rb, d, forcing=mistake != "no_forcing")
        qh = b.copy()
        for _ in range(self.nsmooth[l]):
            qh = qh + self.block_solve(l, self.defect(l, b, Rb, d, qh))
        r = self.defect(l, b, Rb, d, qh)
        b1 = _apply(self.Gam[l], b if mistake == "restrict_b" else qh)
        d1 = _apply(self.Gam[l], r)
        if mistake == "defect_sign":
            d1 = -d1
        y = self.cycle(l + 1, b1, d1, mistake=mistake if mistake == "no_forcing" else None)
        corr = y if mistake == "prolong_y" else y - b1
        qh = qh + _apply(self.Pi[l], corr)
        for _ in range(self.nsmooth[l]):
            qh = qh + self.block_solve(l, self.defect(l, b, Rb, d, qh))
        return qh


def _vortex_case():
    mesh = w.box2d(4, 4, 10.0, 10.0, qg=2, warp=0.1)
    ph = w.Physics(mu=0.01, qinf=w.freestream(2, 0.5))
    X = w.solution_point_coords(mesh, 2)
    q = np.ascontiguousarray(w.isentropic_vortex(X, 5, 5, 5.0, 0.5, 10, 10))
    return mesh, ph, q, [2, 1]


def _omesh_case():
    mesh = w.omesh(6, 12, 0.5, 5.0, 0.02, jitter=0.05, seed=3)
    ph = w.Physics(mu=0.02, qinf=w.freestream(2, 0.3))
    q = angled_flow(mesh, 3, mach=0.3)
    return mesh, ph, q, [3, 2, 1]


@pytest.mark.parametrize("which", ["vortex_p21", "omesh_p321"])
def test_multilevel_cycle_equals_fas_iteration(which):
    mesh, ph, q, levels = _vortex_case() if which == "vortex_p21" else _omesh_case()
    O = oracle.Oracle(mesh, ph, levels)
    dt, nsm_coarse = (0.05, 60) if which == "vortex_p21" else (0.01, 150)
    c = 1.0 / dt + 1.0 / (0.4358665215084590 * dt)
    ids = 1.0 / dt
    L = len(levels)
    nsmooth = [1] * (L - 1) + [nsm_coarse]
    Rq = O.residual(q)
    X = np.random.default_rng(21).standard_normal(q.shape)
    # input scaled so that the correction is ~1e-3 of the state: nonlinear, and the
    # differences R(qh) - R(b) keep about ten significant digits
    X *= 1e-3 * np.abs(q).max() * (c + ids) / np.abs(X).max()
    O.pmg_setup(q, nsmooth, c, ids)
    Y = O.pmg_apply(q, Rq, X)
    # the coarsest level has reached its fixed point: more coarse steps change nothing
    O.pmg_setup(q, nsmooth[:-1] + [nsm_coarse + 20], c, ids)
    Y2 = O.pmg_apply(q, Rq, X)
    assert np.abs(Y2 - Y).max() <= 1e-13 * np.abs(Y).max()    # a few ulps of qh
    ref = FasReference(O, levels, q, nsmooth, c, ids)
    Y_ref = ref.cycle(0, q, X) - q
    err = np.abs(Y - Y_ref).max() / np.abs(Y_ref).max()
    # round-off: the differences R(qh) - R(b) at |qh - b| ~ 1e-3 |q| carry ~1e-13 relative
    # noise, the blocks' conditioning on the stretched mesh a little more
    assert err <= 1e-11, err
    for mistake in ("no_forcing", "restrict_b", "defect_sign", "prolong_y"):
        try:
            bad = ref.cycle(0, q, X, mistake=mistake) - q
        except np.linalg.LinAlgError:       # the planted coarse problem has no solution here
            continue
        e_bad = np.abs(Y - bad).max() / np.abs(Y_ref).max()
        # a planted mistake moves the result by orders of magnitude more than the
        # tolerance (or makes the coarse problem unsolvable: non-finite)
        assert not e_bad <= 1e-6, (mistake, e_bad, err)


def test_two_level_cycle_linearises_to_textbook_two_grid():
    """Small inputs: Y / s -> e2, the linear two-grid iteration with exact coarse solve,
        e0 = M^{-1} X,  e1 = e0 + Pi A1^{-1} Gamma (X - A0 e0),  e2 = e1 + M^{-1} (X - A0 e1),
    A_l = c I - dR_l/dq at (restricted) q, from dense central-difference Jacobians (the
    linear residual of the nonlinear cycle is O(s), here ~1e-7 relative)."""
    mesh, ph, q, levels = _vortex_case()
    O = oracle.Oracle(mesh, ph, levels)
    dt = 0.05
    c = 1.0 / dt + 1.0 / (0.4358665215084590 * dt)
    ids = 1.0 / dt
    nsmooth = [1, 60]
    Rq = O.residual(q)
    X = np.random.default_rng(22).standard_normal(q.shape)
    s = 1e-7 * np.abs(q).max() * (c + ids) / np.abs(X).max()
    O.pmg_setup(q, nsmooth, c, ids)
    Y = O.pmg_apply(q, Rq, s * X) / s
    q1 = O.restrict(q, 0)
    A0 = c * np.eye(q.size) - _dense_jacobian(O, 0, q)
    A1 = c * np.eye(q1.size) - _dense_jacobian(O, 1, q1)
    G1, P1 = oracle.transfer(2, 1)
    Gam, Pi = _kron_d(G1, 2), _kron_d(P1, 2)
    ref = FasReference(O, levels, q, nsmooth, c, ids)
    e0 = ref.block_solve(0, X)
    r0 = X - (A0 @ e0.ravel()).reshape(q.shape)
    ec = np.linalg.solve(A1, _apply(Gam, r0).ravel()).reshape(q1.shape)
    e1 = e0 + _apply(Pi, ec)
    e2 = e1 + ref.block_solve(0, X - (A0 @ e1.ravel()).reshape(q.shape))
    err = np.abs(Y - e2).max() / np.abs(e2).max()
    assert err <= 1e-5, err
    # the coarse correction matters at this tolerance
    e_no_coarse = e0 + ref.block_solve(0, X - (A0 @ e0.ravel()).reshape(q.shape))
    assert np.abs(Y - e_no_coarse).max() / np.abs(e2).max() > 1e-2
