"""Pins of the oracle's FR operator tables and p-transfer operators (Sec. 2.1; Eqs. 17-18).

Each check compares against something other than the oracle itself: numpy's
Gauss-Legendre / Legendre routines, exactness on polynomials, closed forms of the DG
correction functions, and the defining properties of an L2 projection."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

import oracle


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_gauss_legendre_matches_numpy(p):
    t = oracle.table(p)
    x, w = npleg.leggauss(p + 1)
    assert np.allclose(t["x"], x, rtol=0, atol=2e-16)
    assert np.allclose(t["w"], w, rtol=0, atol=4e-16)
    # quadrature exact to degree 2p+1
    for k in range(2 * p + 2):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.dot(t["w"], t["x"] ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_derivative_and_interpolation_exact_on_polynomials(p):
    t = oracle.table(p)
    x = t["x"]
    for k in range(p + 1):
        f = x ** k
        df = k * x ** (k - 1) if k else 0 * x
        assert np.allclose(t["D"] @ f, df, atol=1e-12)
        assert abs(t["lm"] @ f - (-1.0) ** k) < 1e-13
        assert abs(t["lp"] @ f - 1.0) < 1e-13
        dm = k * (-1.0) ** (k - 1) if k else 0.0
        assert abs(t["dlm"] @ f - dm) < 1e-12
        assert abs(t["dlp"] @ f - (k if k else 0.0)) < 1e-12
    # rows of D sum to zero exactly up to rounding; middle node of odd n is exactly 0
    assert np.allclose(t["D"].sum(axis=1), 0, atol=1e-13)
    if (p + 1) % 2 == 1:
        assert t["x"][p // 2] == 0.0


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_correction_functions_closed_form(p):
    t = oracle.table(p)
    # g_L = (-1)^p/2 (P_p - P_{p+1}); g_R = (P_p + P_{p+1})/2 -> derivatives through numpy
    cp = np.zeros(p + 2); cp[p] = 1
    cq = np.zeros(p + 2); cq[p + 1] = 1
    gL = (-1) ** p / 2 * (cp - cq)
    gR = (cp + cq) / 2
    dgL, dgR = npleg.legder(gL), npleg.legder(gR)
    assert np.allclose(t["gLd"], npleg.legval(t["x"], dgL), atol=1e-12)
    assert np.allclose(t["gRd"], npleg.legval(t["x"], dgR), atol=1e-12)
    # closed forms at the faces: g_L'(-1) = -(p+1)^2/2, g_R'(1) = (p+1)^2/2
    assert t["gLf"] == -((p + 1) ** 2) / 2
    assert t["gRf"] == ((p + 1) ** 2) / 2
    # end values g_L(-1) = 1, g_L(1) = 0
    assert abs(npleg.legval(-1, gL) - 1) < 1e-14 and abs(npleg.legval(1, gL)) < 1e-14
    # DG recovery: g_R' at the nodes equals l_i(1) / w_i (lifting through the GL mass matrix)
    assert np.allclose(t["gRd"], t["lp"] / t["w"], atol=1e-12)


@pytest.mark.parametrize("p0,p1", [(2, 1), (3, 2), (3, 1), (4, 2), (2, 1), (4, 3), (3, 3)])
def test_transfer_operators(p0, p1):
    G, P = oracle.transfer(p0, p1)
    # Gamma o Pi = identity on P^{p1}
    assert np.allclose(G @ P, np.eye(p1 + 1), atol=1e-15)
    t0, t1 = oracle.table(p0), oracle.table(p1)
    # Pi interpolates any degree-p1 polynomial exactly onto the p0 nodes
    for k in range(p1 + 1):
        assert np.allclose(P @ t1["x"] ** k, t0["x"] ** k, atol=1e-14)
    # Gamma is the L2 projection: residual orthogonal to P^{p1} (fine quadrature from numpy)
    xq, wq = npleg.leggauss(12)
    rng = np.random.default_rng(p0 * 10 + p1)
    f0 = rng.standard_normal(p0 + 1)

    def lag(xs, vals, y):
        out = np.zeros_like(y)
        for i in range(len(xs)):
            li = np.ones_like(y)
            for k in range(len(xs)):
                if k != i:
                    li *= (y - xs[k]) / (xs[i] - xs[k])
            out += vals[i] * li
        return out
    f1 = G @ f0
    r = lag(t0["x"], f0, xq) - lag(t1["x"], f1, xq)
    for k in range(p1 + 1):
        assert abs(np.sum(wq * r * xq ** k)) < 1e-14
