"""Basis functions and the prolongation operator P of Sec. 3.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Basis operators (Eqs. 8-11), each multiplied row-wise by V_i (and by rho_i
for the rho-weighted ones, which does not change the local solutions):
  (B1)  c^nu Phi - (1/rho^nu) div(rho^nu lambda grad Phi) = 0
        -> A_b = diag(V rho^nu c^nu) + rho_f-weighted TPFA Laplacian
  (B2)  -(1/rho^nu) div(rho^nu lambda grad Phi) = 0
        -> A_b = rho_f-weighted TPFA Laplacian
  (B3)  c^n Phi - div(lambda grad Phi) = 0
        -> A_b = diag(V c^n) + TPFA Laplacian, c^n = Eq. 4 at p = p^n
  (B4)  -div(lambda grad Phi) = 0
        -> A_b = TPFA Laplacian
Reading R10: A_b holds internal faces only; the global Dirichlet faces and
the sources do not enter the local problems, whose boundary conditions are
the reduced-problem (localisation) conditions.
Reading R19: prescribed-pressure cells are eliminated from A_b as from A
(unit rows, no couplings; free rows keep their diagonal), so the local
problems see a homogeneous Dirichlet condition there and the basis values
of a fixed cell are zero.

Reading R9 (the paper cites the algebraic multiscale solver for the
reduced-problem conditions without restating them): wirebasket construction.
With the fine cells split by level (see wirebasket.py), the basis values of
level-k cells solve, entity by entity,
    M_e P_e = - A_b[e, lower] P[lower],
    M_e = A_b[e, e] + diag(sum of A_b[i, j] over neighbours j of level k+1),
where "lower" are the neighbouring cells of level k-1 (already known) and
vertex cells carry P[v, J(v)] = 1.  Level-(k+1) neighbours are thus lumped
onto the diagonal (no flux across the entity), which for a zero-row-sum
A_b reproduces a partition of unity.  The highest level (dual-block
interiors) has no such neighbours.  P is N_f x N_c with basis function
Phi_k in column k (Eq. 12).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .problem import Problem, accumulation_coefficient, eliminate_fixed
from .wirebasket import Wirebasket


def basis_operator(pb: Problem, kind: int, rho_nu, c_nu, p_n, dt) -> sp.csr_matrix:
    """A_b of Eqs. 8-11 (see module docstring) as a CSR matrix."""
    g, fc, fl = pb.grid, pb.faces, pb.fluid
    N, V = g.N, g.V
    if kind in (1, 2):
        w = fc.T * (0.5 * (rho_nu[fc.lo] + rho_nu[fc.hi]))
    elif kind in (3, 4):
        w = fc.T.copy()
    else:
        raise ValueError("basis kind must be 1..4")
    if kind == 1:
        dg = V * rho_nu * c_nu
    elif kind == 3:
        dg = V * accumulation_coefficient(fl, p_n, p_n, dt)
    else:
        dg = np.zeros(N)
    rows = np.concatenate([fc.lo, fc.hi, fc.lo, fc.hi, np.arange(N)])
    cols = np.concatenate([fc.lo, fc.hi, fc.hi, fc.lo, np.arange(N)])
    vals = np.concatenate([w, w, -w, -w, dg])
    Ab = sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()
    Ab.sum_duplicates()
    Ab.sort_indices()
    if pb.has_fixed:
        Ab = eliminate_fixed(Ab, pb.fixed)
    return Ab


class PRows:
    """Row storage of P: for every fine cell up to 8 (coarse id, value)
    pairs.  Each fine cell is covered by at most the 2^3 vertices spanning
    its dual block, so 8 slots always suffice."""

    def __init__(self, N):
        self.col = np.full((N, 8), -1, np.int64)
        self.val = np.zeros((N, 8))

    def set_rows(self, cells, corners, values):
        k = len(corners)
        self.col[cells, :] = -1
        self.val[cells, :] = 0.0
        self.col[cells, :k] = corners[None, :]
        self.val[cells, :k] = values

    def dense_rows(self, cells, corners):
        """P[cells][:, corners] as a dense array."""
        out = np.zeros((len(cells), len(corners)))
        cc = self.col[cells]
        vv = self.val[cells]
        for s in range(8):
            m = cc[:, s] >= 0
            if not np.any(m):
                continue
            pos = np.searchsorted(corners, cc[m, s])
            ok = (pos < len(corners))
            ok[ok] = corners[pos[ok]] == cc[m, s][ok]
            if not np.all(ok):
                raise AssertionError("a lower-level neighbour carries a basis function "
                                     "that is not a corner of this entity")
            out[np.nonzero(m)[0], pos] += vv[m, s]
        return out

    def to_csr(self, Nc):
        N = self.col.shape[0]
        r = np.repeat(np.arange(N), 8)
        c = self.col.ravel()
        v = self.val.ravel()
        m = c >= 0
        return sp.csr_matrix((v[m], (r[m], c[m])), shape=(N, Nc))


def solve_entity(Ab: sp.csr_matrix, wb: Wirebasket, P: PRows, e):
    """Reduced-problem solve of one entity (edge, face or interior)."""
    M, rhs = entity_system(Ab, wb, P, e)
    return np.linalg.solve(M, rhs)


def entity_system(Ab: sp.csr_matrix, wb: Wirebasket, P: PRows, e):
    """The dense local matrix M_e and right-hand sides of one entity."""
    S = e.cells
    k = e.level
    m = len(S)
    sub = Ab[S].tocoo()
    r, c, v = sub.row, sub.col, sub.data
    pos = np.full(Ab.shape[0], -1, np.int64)
    pos[S] = np.arange(m)
    inS = pos[c] >= 0
    lev = wb.level[c]
    if np.any((~inS) & (lev == k)):
        raise AssertionError("entity touches another entity of its own level")
    M = np.zeros((m, m))
    np.add.at(M, (r[inS], pos[c[inS]]), v[inS])
    up = (~inS) & (lev == k + 1)
    M[np.arange(m), np.arange(m)] += np.bincount(r[up], weights=v[up], minlength=m)
    lo = (~inS) & (lev == k - 1)
    Plo = P.dense_rows(c[lo], e.corners)                # rows aligned with the lo entries
    rhs = np.zeros((m, len(e.corners)))
    np.add.at(rhs, r[lo], -v[lo][:, None] * Plo)
    return M, rhs


def prolongation(Ab: sp.csr_matrix, wb: Wirebasket, P: PRows | None = None,
                 rebuild=None) -> PRows:
    """Staged construction vertex -> edge -> face -> interior.

    rebuild: optional boolean per entity; entities not flagged keep their
    rows of the given P (used by the adaptive update of Sec. 4.1.2)."""
    N = wb.grid.N
    if P is None:
        P = PRows(N)
    J = np.arange(wb.Nc)
    P.set_rows(wb.vertex_cell, np.zeros(0, np.int64), np.zeros((wb.Nc, 0)))
    P.col[wb.vertex_cell, 0] = J
    P.val[wb.vertex_cell, 0] = 1.0
    for k in range(1, wb.d_active + 1):
        for ei, e in enumerate(wb.entities):
            if e.level != k or (rebuild is not None and not rebuild[ei]):
                continue
            P.set_rows(e.cells, e.corners, solve_entity(Ab, wb, P, e))
    return P


def prolongation_global(Ab: sp.csr_matrix, wb: Wirebasket) -> sp.csr_matrix:
    """Independent route to the same P: assemble the whole block-triangular
    reduced system in the natural cell order and solve it at once.

    Row i of level k keeps A_b[i, j] for neighbours j of level k and k-1,
    lumps the level-(k+1) neighbours onto its diagonal, and vertex rows are
    identity rows; the right-hand side is the vertex indicator matrix."""
    N = wb.grid.N
    coo = Ab.tocoo()
    r, c, v = coo.row, coo.col, coo.data
    lr, lc = wb.level[r], wb.level[c]
    keep = (r != c) & ((lc == lr) | (lc == lr - 1)) & (lr > 0)
    lump = (r != c) & (lc == lr + 1) & (lr > 0)
    diag = np.where(wb.level > 0, Ab.diagonal(), 1.0)
    diag = diag + np.bincount(r[lump], weights=v[lump], minlength=N)
    rows = np.concatenate([r[keep], np.arange(N)])
    cols = np.concatenate([c[keep], np.arange(N)])
    vals = np.concatenate([v[keep], diag])
    red = sp.csc_matrix((vals, (rows, cols)), shape=(N, N))
    E = sp.csc_matrix((np.ones(wb.Nc), (wb.vertex_cell, np.arange(wb.Nc))), shape=(N, wb.Nc))
    return sp.csr_matrix(spl.spsolve(red, E))


def correction_function(Ab: sp.csr_matrix, wb: Wirebasket, r: np.ndarray) -> np.ndarray:
    """Correction function Psi (Sec. 3: the local problems of Eqs. 8-11 with
    their right-hand side kept; Table 1, step 4, the pre-smoothing stage).

    Reading R21: the same reduced problems as the basis functions, with the
    fine-scale residual r as the source: Psi = 0 on the vertices, then level
    by level (edges, faces, interiors) M_e Psi_e = r_e - A_b[e, lower] Psi[lower],
    M_e = A_b[e, e] with the level-(k+1) neighbours lumped onto the diagonal."""
    psi = np.zeros(wb.grid.N)
    for k in range(1, wb.d_active + 1):
        for e in wb.entities:
            if e.level != k:
                continue
            S = e.cells
            m = len(S)
            sub = Ab[S].tocoo()
            rr, c, v = sub.row, sub.col, sub.data
            pos = np.full(Ab.shape[0], -1, np.int64)
            pos[S] = np.arange(m)
            inS = pos[c] >= 0
            lev = wb.level[c]
            M = np.zeros((m, m))
            np.add.at(M, (rr[inS], pos[c[inS]]), v[inS])
            up = (~inS) & (lev == k + 1)
            M[np.arange(m), np.arange(m)] += np.bincount(rr[up], weights=v[up], minlength=m)
            lo = (~inS) & (lev == k - 1)
            rhs = np.array(r[S], dtype=np.float64)
            np.add.at(rhs, rr[lo], -v[lo] * psi[c[lo]])
            psi[S] = np.linalg.solve(M, rhs)
    return psi
