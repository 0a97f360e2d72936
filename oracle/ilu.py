"""ILU(0), the fine-scale second-stage smoother of Sec. 3 and Table 1
(step 6), here written for a general sparse matrix.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading R12: unknowns are taken in the natural (lexicographic) order of the
fine cells, without pivoting.  The factors keep exactly the sparsity pattern
of A: L is unit lower triangular and U upper triangular with (L U)_ij = a_ij
for every (i, j) in the pattern of A.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def ilu0(A: sp.csr_matrix):
    """Row-by-row (IKJ) incomplete LU restricted to the pattern of A.

    For each row i, for each k < i in the row (ascending):
        a_ik <- a_ik / a_kk
        a_ij <- a_ij - a_ik a_kj   for every j > k present in both rows.
    Returns (L, U) as CSR matrices."""
    A = sp.csr_matrix(A, copy=True)
    A.sort_indices()
    n = A.shape[0]
    ip, ix = A.indptr, A.indices
    a = A.data.astype(np.float64).tolist()
    ixl = ix.tolist()
    ipl = ip.tolist()
    diag_pos = [0] * n
    for i in range(n):
        s, e = ipl[i], ipl[i + 1]
        for q in range(s, e):
            if ixl[q] == i:
                diag_pos[i] = q
                break
        else:
            raise ZeroDivisionError(f"row {i} has no diagonal entry")
    for i in range(n):
        s, e = ipl[i], ipl[i + 1]
        where = {ixl[q]: q for q in range(s, e)}
        for q in range(s, e):
            k = ixl[q]
            if k >= i:
                break
            a[q] = a[q] / a[diag_pos[k]]
            lik = a[q]
            for qq in range(diag_pos[k] + 1, ipl[k + 1]):
                j = ixl[qq]
                t = where.get(j)
                if t is not None:
                    a[t] -= lik * a[qq]
        if a[diag_pos[i]] == 0.0:
            raise ZeroDivisionError(f"zero pivot in row {i}")
    F = sp.csr_matrix((np.asarray(a), ix.copy(), ip.copy()), shape=A.shape)
    L = sp.tril(F, k=-1, format="csr") + sp.identity(n, format="csr")
    U = sp.triu(F, k=0, format="csr")
    return L.tocsr(), U.tocsr()


def ilu_apply(LU, r: np.ndarray) -> np.ndarray:
    """M^{-1} r with M = L U: forward then backward substitution."""
    L, U = LU
    w = spl.spsolve_triangular(L, r, lower=True, unit_diagonal=True)
    return spl.spsolve_triangular(U, w, lower=False)
