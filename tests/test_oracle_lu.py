"""Pins of the oracle's dense LU (the element-Jacobi smoother's factor/solve): against
numpy's LAPACK solve on random and pivoting-heavy matrices, and the factor layout
(unit L below, U above, 1/u_kk on the diagonal) against a product that rebuilds P A."""
import ctypes as C

import numpy as np
import pytest

import oracle


def _lu(A):
    n = A.shape[0]
    F = np.ascontiguousarray(A, dtype=np.float64).copy()
    piv = np.zeros(n, dtype=np.int32)
    oracle.lib().or_lu_factor(n, F.ctypes.data_as(C.POINTER(C.c_double)), piv.ctypes.data_as(C.POINTER(C.c_int)))
    return F, piv


def _solve(F, piv, b):
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    oracle.lib().or_lu_solve(F.shape[0], F.ctypes.data_as(C.POINTER(C.c_double)),
                             piv.ctypes.data_as(C.POINTER(C.c_int)), x.ctypes.data_as(C.POINTER(C.c_double)))
    return x


@pytest.mark.parametrize("n", [1, 5, 36, 100])
def test_solve_matches_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.1
    b = rng.standard_normal(n)
    F, piv = _lu(A)
    x = _solve(F, piv, b)
    ref = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    assert np.abs(x - ref).max() <= 1e-15 * cond * np.abs(ref).max() * 10


def test_factor_layout_rebuilds_permuted_matrix():
    rng = np.random.default_rng(7)
    n = 12
    A = rng.standard_normal((n, n))
    A[0, 0] = 1e-14          # forces a row swap at the first step
    F, piv = _lu(A)
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F, 1) + np.diag(1.0 / np.diag(F))
    PA = A.copy()
    for k in range(n):       # the factor's swaps, in order
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    assert piv[0] != 0
    assert np.abs(L @ U - PA).max() <= 1e-13 * np.abs(A).max()
    # every multiplier is bounded by 1 (partial pivoting)
    assert np.abs(np.tril(F, -1)).max() <= 1.0


def _solve_div(A, b):
    n = A.shape[0]
    F = np.ascontiguousarray(A, dtype=np.float64).copy()
    piv = np.zeros(n, dtype=np.int32)
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    L = oracle.lib()
    L.or_lu_factor_div(n, F.ctypes.data_as(C.POINTER(C.c_double)), piv.ctypes.data_as(C.POINTER(C.c_int)))
    L.or_lu_solve_div(n, F.ctypes.data_as(C.POINTER(C.c_double)), piv.ctypes.data_as(C.POINTER(C.c_int)),
                      x.ctypes.data_as(C.POINTER(C.c_double)))
    return x


@pytest.mark.parametrize("which,shifts", [("unsteady_p3", (1e-2, 1.0, 1e2)),
                                          ("steady_p4", (1e-4, 1e-2, 1.0, 1e2))])
def test_reciprocal_pivots_agree_with_division_on_wall_blocks(which, shifts):
    """The factor keeps 1/u_kk and the backward substitution multiplies; the textbook form
    divides by u_kk.  On the element blocks of the wall rings of stretched cylinder O-meshes
    (Ma 0.05, p = 3: condition numbers ~1e7; Ma 1e-3, p = 4 at the impulsive start: ~1e15
    in the conservative variables), for the pseudo-time shifts the solvers use, the two
    forms give the same solutions to 1e-12 (max norm, relative): one rounding per unknown
    of the backward substitution, amplified by the triangular factor, stays far below it."""
    from paper_2202_09733_gb300 import workloads as w
    W = (w.cylinder_unsteady(nr=6, nt=12, p=3, levels=[3]) if which == "unsteady_p3"
         else w.cylinder_steady(nr=6, nt=12, p=4, levels=[4]))
    O = oracle.Oracle(W.mesh, W.phys, W.levels)
    rng = np.random.default_rng(11)
    wall = np.arange(12)                       # the first radial ring touches the wall
    kmax = 0.0
    for shift in shifts:
        for Me in O.elem_blocks(W.q0, shift, wall):
            b = Me @ rng.standard_normal(Me.shape[0])
            F, piv = _lu(Me)
            x_rec = _solve(F, piv, b)
            x_div = _solve_div(Me, b)
            assert np.abs(x_rec - x_div).max() <= 1e-12 * np.abs(x_div).max()
            kmax = max(kmax, np.linalg.cond(Me))
    assert kmax > (1e6 if which == "unsteady_p3" else 1e12)    # the blocks are ill-conditioned
