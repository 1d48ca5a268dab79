"""Pins of the oracle's p-adaptation indicator, marking and nested hierarchies (Sec. 3.3).

- eta = 0 for a field in Q^{p-1} (monomials, not Legendre polynomials, so the basis of
  the check is not the indicator's own);
- eta = 1 for the pure top mode phi_p(xi) phi_0(eta);
- s = 1 + xi^p on [-1, 1]^2: eta in closed form from the leading coefficient of P_p;
- brute force: the L2 projection onto Q^{p-1} by least squares over monomials with a
  finer quadrature of the nodal interpolant, in 2-D and 3-D, for random fields;
- eta is invariant under scaling and reads the named variable;
- the marking rule and the bounds, by hand; the hierarchy rule against the paper's eight
  examples."""
import math

import numpy as np
import pytest

from oracle import padapt as PA


def _state(field, d, p, E=1, nv=5, var=1):
    """A state [nv][Np][E] whose variable var holds field(xi, eta[, zeta]) at the GL
    points (the index of the first coordinate runs fastest)."""
    xi, _ = np.polynomial.legendre.leggauss(p + 1)
    grids = np.meshgrid(*([xi] * d), indexing="ij")[::-1]   # last axis fastest -> x fastest
    vals = field(*grids).reshape(-1)
    q = np.zeros((nv, (p + 1) ** d, E))
    q[var, :, :] = vals[:, None]
    return q


@pytest.mark.parametrize("d,p", [(2, 1), (2, 3), (2, 4), (3, 2), (3, 3)])
def test_lower_degree_fields_have_zero_indicator(d, p):
    rng = np.random.default_rng(d * 10 + p)
    coef = rng.standard_normal((p,) * d)

    def f(*x):
        out = np.zeros_like(x[0])
        for idx in np.ndindex(*coef.shape):
            term = coef[idx]
            for ax, k in enumerate(idx):
                term = term * x[ax] ** k
            out = out + term
        return out
    eta = PA.spectral_decay(_state(f, d, p), d, p)
    assert eta[0] <= 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_top_mode_has_unit_indicator(p):
    _, _, Phi = PA.legendre_modes(p)
    c = np.zeros(p + 1)
    c[p] = 1.0
    f = lambda x, y: np.polynomial.legendre.legval(x, c) * (1.0 + 0.0 * y)
    eta = PA.spectral_decay(_state(f, 2, p), 2, p)
    assert abs(eta[0] - 1.0) <= 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_one_plus_xi_to_the_p_closed_form(p):
    # xi^p = phi_p / (sqrt((2p+1)/2) k_p) + lower degrees, k_p = (2p)! / (2^p (p!)^2)
    k_p = math.factorial(2 * p) / (2 ** p * math.factorial(p) ** 2)
    c_p = 1.0 / (math.sqrt((2 * p + 1) / 2.0) * k_p)
    removed2 = 2.0 * c_p ** 2                                   # times int over eta of 1
    total2 = 2.0 * (2.0 + (4.0 / (p + 1) if p % 2 == 0 else 0.0) + 2.0 / (2 * p + 1))
    eta_ref = math.sqrt(removed2 / total2)
    eta = PA.spectral_decay(_state(lambda x, y: 1.0 + x ** p, 2, p), 2, p)
    assert abs(eta[0] - eta_ref) <= 1e-13 * max(1.0, eta_ref)


def _brute_force(values, d, p):
    """||s - P s|| / ||s|| with P the L2 projection onto Q^{p-1}, by least squares over
    monomials on a (p + 3)-point Gauss rule of the nodal interpolant of s."""
    xi, _ = np.polynomial.legendre.leggauss(p + 1)
    xf, wf = np.polynomial.legendre.leggauss(p + 3)
    # 1-D Lagrange basis of the GL nodes at the fine points: L[f, i]
    L = np.ones((len(xf), p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            if j != i:
                L[:, i] *= (xf - xi[j]) / (xi[i] - xi[j])
    s = values.reshape((p + 1,) * d)                    # axes (.., y, x): x fastest
    for ax in range(d):
        s = np.moveaxis(np.tensordot(L, s, axes=([1], [ax])), 0, ax)
    grids = np.meshgrid(*([xf] * d), indexing="ij")[::-1]
    W = np.ones_like(grids[0])
    for g in np.meshgrid(*([wf] * d), indexing="ij"):
        W = W * g
    cols = []
    for idx in np.ndindex(*((p,) * d)):
        term = np.ones_like(grids[0])
        for ax, k in enumerate(idx):
            term = term * grids[ax] ** k
        cols.append(term.reshape(-1))
    B = np.stack(cols, axis=1)
    sw = np.sqrt(W.reshape(-1))
    sv = s.reshape(-1)
    coef, *_ = np.linalg.lstsq(B * sw[:, None], sv * sw, rcond=None)
    r = sv - B @ coef
    return math.sqrt(np.sum(W.reshape(-1) * r * r) / np.sum(W.reshape(-1) * sv * sv))


@pytest.mark.parametrize("d,p", [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3)])
def test_random_fields_against_brute_force_projection(d, p):
    rng = np.random.default_rng(100 + d * 10 + p)
    E = 4
    q = rng.standard_normal((5, (p + 1) ** d, E))
    eta = PA.spectral_decay(q, d, p, var=1)
    for e in range(E):
        assert abs(eta[e] - _brute_force(q[1, :, e], d, p)) <= 1e-12


def test_scaling_invariance_and_variable():
    rng = np.random.default_rng(7)
    q = rng.standard_normal((5, 16, 3))
    e1 = PA.spectral_decay(q, 2, 3, var=1)
    q2 = q.copy()
    q2[1] *= -37.5
    q2[2] += 100.0                                       # another variable: no effect
    assert np.allclose(PA.spectral_decay(q2, 2, 3, var=1), e1, rtol=1e-13, atol=0)
    assert not np.allclose(PA.spectral_decay(q, 2, 3, var=2), e1)
    assert PA.spectral_decay(np.zeros((5, 16, 2)), 2, 3)[0] == 0.0


def test_marking_rule_by_hand():
    eta = np.array([1.0, 0.5, 0.1, 1e-4, 0.3, 5e-4])
    p = np.array([3, 3, 3, 3, 4, 1])
    out = PA.mark(eta, p, p_min=1, p_max=4)
    # eta_max = 1: raise where eta > 0.2, lower where eta < 1e-3, within [1, 4]
    assert out.tolist() == [4, 4, 3, 2, 4, 1]


def test_nested_hierarchies_match_the_papers_examples():
    assert [PA.nested_hierarchy(p, 1, 3) for p in (4, 3, 2, 1)] == [[4, 3, 2], [3, 2, 1], [2, 1, 0], [1, 0, 0]]
    assert [PA.nested_hierarchy(p, 2, 3) for p in (4, 3, 2, 1)] == [[4, 2, 0], [3, 1, 0], [2, 1, 0], [1, 0, 0]]


def test_library_hierarchy_rule_equals_the_oracle():
    """The library's host rule (fr_nested_hierarchy, no GPU needed) against the oracle's."""
    from paper_2202_09733_gb300 import api
    for p in range(0, 6):
        for gap in (1, 2, 3):
            for nl in (1, 2, 3, 4):
                assert api.fr_nested_hierarchy(p, gap, nl) == PA.nested_hierarchy(p, gap, nl), (p, gap, nl)
