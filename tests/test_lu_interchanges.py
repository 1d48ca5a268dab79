"""The row-interchange bookkeeping of the phased (tensor-core) block LU, checked on the
CPU in float64 against LAPACK's LU with partial pivoting (scipy.linalg.lu_factor).

The GPU factorisation eliminates in 32-column panels over the whole batch and applies a
panel's interchanges to the trailing columns only (as a gather of the rows), leaving the
columns of L left of the panel alone until a final pass.  Its correctness rests on three
facts that this test restates in numpy and checks on random matrices that need pivoting:
  - composing the panel's transpositions tau_c = (k0 + c, p_c), p_c >= k0 + c, as a gather
    gives src(i) = tau_0(tau_1(... tau_31(i))), and for a row i below the panel src(i)
    is i or a panel row (so a trailing tile can read its lower rows where they are);
  - the final pass moves panel j's L columns by pi_j = the later panels' interchanges
    composed the same way, and the overall permutation is perm = pi_{-1};
  - the result equals LAPACK's factors and pivot rows (first maximal |a|)."""
import numpy as np
import pytest
import scipy.linalg as sla

NB = 32


def compose(piv, k0, n, x):
    """x after the interchanges (k0 + t, piv[k0 + t]), t = 0 .. n-1, read as a gather."""
    for t in range(n - 1, -1, -1):
        a, b = k0 + t, piv[k0 + t]
        x = b if x == a else (a if x == b else x)
    return x


def phased_lu(A):
    """The GPU algorithm's arithmetic in float64 on one block (column-major semantics kept
    in numpy's row/column indexing): panel by panel, trailing gathers, final L pass."""
    A = A.copy()
    nd = A.shape[0]
    piv = np.arange(nd)
    for k0 in range(0, nd, NB):
        kb = min(NB, nd - k0)
        # panel: partial pivoting inside the panel columns, whole panel rows interchanged
        for c in range(kb):
            k = k0 + c
            col = np.abs(A[k:, k])
            p = k + int(np.argmax(col))            # first maximal |a|
            piv[k] = p
            if p != k:
                A[[k, p], k0:k0 + kb] = A[[p, k], k0:k0 + kb]
            A[k + 1:, k] /= A[k, k]
            A[k + 1:, k + 1:k0 + kb] -= np.outer(A[k + 1:, k], A[k, k + 1:k0 + kb])
        r0 = k0 + kb
        if r0 >= nd:
            break
        # trailing columns: rows gathered in the panel's interchange order
        src = [compose(piv, k0, kb, k0 + i) for i in range(nd - k0)]
        for i in range(kb, nd - k0):              # rows below the panel: itself or a panel row
            assert src[i] == k0 + i or k0 <= src[i] < r0
        T = A[src, r0:].copy()
        L11 = np.tril(A[k0:r0, k0:r0], -1) + np.eye(kb)
        U12 = np.linalg.solve(L11, T[:kb])
        A[k0:r0, r0:] = U12
        A[r0:, r0:] = T[kb:] - A[r0:, k0:r0] @ U12
    # final pass: panel j's L columns take the later panels' interchanges
    np_ = (nd + NB - 1) // NB
    for j in range(np_ - 1):
        k0, r1 = j * NB, (j + 1) * NB
        pij = [x for x in range(nd)]
        for x in range(r1, nd):
            y = x
            for jj in range(np_ - 1, j, -1):
                kk0 = jj * NB
                y = compose(piv, kk0, min(NB, nd - kk0), y)
            pij[x] = y
        A[r1:, k0:r1] = A[[pij[x] for x in range(r1, nd)], k0:r1]
    perm = []
    for x in range(nd):
        y = x
        for jj in range(np_ - 1, -1, -1):
            kk0 = jj * NB
            y = compose(piv, kk0, min(NB, nd - kk0), y)
        perm.append(y)
    return A, piv, np.array(perm)


@pytest.mark.parametrize("nd,seed", [(100, 0), (135, 1), (160, 2)])
def test_phased_lu_equals_lapack(nd, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((nd, nd))
    F, piv, perm = phased_lu(A)
    lu, lp = sla.lu_factor(A)
    assert np.array_equal(piv, lp)                       # the same pivot rows
    assert np.max(np.abs(F - lu)) <= 1e-10 * np.max(np.abs(lu))
    # perm[i] = the row of A now at row i: P A = L U
    L = np.tril(F, -1) + np.eye(nd)
    U = np.triu(F)
    assert np.max(np.abs(A[perm] - L @ U)) <= 1e-12 * nd * np.max(np.abs(A))
    assert (piv != np.arange(nd)).any()
