"""Restriction, coarse-scale operator and coarse solve of Sec. 3.

TEST INFRASTRUCTURE ONLY (see the package docstring).

  MSFE:  R = P^T                                   (Sec. 3)
  MSFV:  R(i, j) = 1 iff fine cell j lies in primal block i   (Eq. 7)
  coarse system  (R A P) p_c = R f                 (Eq. 13)
  residual form  dp' = P (R A P)^{-1} R r          (Eq. 15)
The coarse matrix is formed with the full fine matrix A (accumulation and
Dirichlet terms included) and factorised by dense LU with partial pivoting.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .wirebasket import Wirebasket


def restriction(kind: int, P: sp.csr_matrix, wb: Wirebasket) -> sp.csr_matrix:
    if kind == 0:
        return sp.csr_matrix(P.T)
    g = wb.grid
    x, y, z = g.coords()
    bx, by, bz = wb.coarse
    I = (x // bx) + wb.nc[0] * ((y // by) + wb.nc[1] * (z // bz))
    return sp.csr_matrix((np.ones(g.N), (I, np.arange(g.N))), shape=(wb.Nc, g.N))


def coarse_operator(R: sp.csr_matrix, A: sp.csr_matrix, P: sp.csr_matrix) -> np.ndarray:
    """A_c = R A P (Eq. 13) as a dense N_c x N_c array."""
    return (R @ (A @ P)).toarray()


def coarse_factor(Ac: np.ndarray):
    return sla.lu_factor(Ac)


def coarse_solve(lu, rc: np.ndarray) -> np.ndarray:
    return sla.lu_solve(lu, rc)
