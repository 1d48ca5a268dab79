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
