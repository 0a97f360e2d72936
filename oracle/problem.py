"""Fine-scale problem of Sec. 2: single-phase compressible flow, Eq. 1
(mass), its implicit-Euler form Eq. 2 (p-nonlinear), the Newton
linearisation Eqs. 3-5 (lin_p, p_lhs, p_rhs), the algebraic system Eq. 6
(ap=r) and the nonlinear error Eq. 19 (epsilon_nu).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions
-----------
Cartesian grid, cell index i = x + nx*(y + ny*z).  A direction with a single
cell is inactive (2D when nz = 1).  Permeability is a diagonal tensor
(kx, ky, kz) per cell, mobility lambda = k / mu.

Reading R2 (the paper only says "finite-volume transmissibilities"): two-point
flux approximation with the harmonic average of the two half-cell
conductances on internal faces, and a half-cell distance to the Dirichlet
face value on west/east boundary faces.
Reading R3: constant porosity (d phi / dp = 0).
Reading R4: face density is the arithmetic mean of the two cell densities;
on a Dirichlet face it is rho(p_boundary).
Reading R6: the saturation S^n of Eq. 19 is 1 (single phase).
Reading R7: every row of Eq. 3 is multiplied by V_i rho_i^nu, which makes the
matrix A = C + A~ of Eq. 6 symmetric and leaves its solution unchanged.
Reading R22 (the full-Jacobian variant; the paper's own step is Eq. 3):
Newton on the paper's equation (Eq. 2 divided by rho, in volume units) with
every term differentiated, the flux density and the flux term's 1/rho
included, and rows multiplied by V rho^nu as in R7.  Both steps solve
A dp = -F(p^nu) for the same residual F, so they share the root.
Reading R19 (Test Case 2 of Sec. 4.2.2 prescribes p at the centres of two
vertical columns of cells without saying how): the prescribed ("fixed") cells
are taken out of the unknowns by symmetric elimination.  Their entries of
the iterate hold the prescribed values, each fixed row of A reads
p_i = p_D (unit diagonal, no couplings), the couplings of free cells to
fixed cells move to the right-hand side, and Eq. 19 is not imposed at fixed
cells (eps = 0 there).  A fixed cell may not be a coarse node: eliminating
it would remove a coarse unknown.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def V(self) -> float:
        return self.dx * self.dy * self.dz

    def coords(self):
        i = np.arange(self.N)
        return i % self.nx, (i // self.nx) % self.ny, i // (self.nx * self.ny)


@dataclass(frozen=True)
class Fluid:
    """law 0: rho = rho0 exp(c p) ; law 1: rho = rho0 (1 + eta p) (Sec. 4)."""
    law: int = 0
    c_or_eta: float = 0.1
    rho0: float = 1.0
    mu: float = 1.0
    phi: float = 0.1

    def rho(self, p):
        if self.law == 0:
            return self.rho0 * np.exp(self.c_or_eta * p)
        return self.rho0 * (1.0 + self.c_or_eta * p)

    def drho(self, p):
        if self.law == 0:
            return self.c_or_eta * self.rho0 * np.exp(self.c_or_eta * p)
        return self.rho0 * self.c_or_eta * np.ones_like(p)


@dataclass(frozen=True)
class BC:
    """Dirichlet pressure on the west (x = 0) and east (x = nx-1) faces, or
    none (no-flow everywhere); plus point sources with volumetric rates
    Q_i = q_i dV_i (the integrated source of Eq. 6), positive = injection;
    plus cells whose centre pressure is prescribed (Reading R19)."""
    dirichlet: bool = True
    p_west: float = 1.0
    p_east: float = 0.0
    src_cell: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    src_rate: np.ndarray = field(default_factory=lambda: np.zeros(0))
    fix_cell: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    fix_value: np.ndarray = field(default_factory=lambda: np.zeros(0))

    def source_vector(self, N):
        Q = np.zeros(N)
        np.add.at(Q, np.asarray(self.src_cell, dtype=np.int64), np.asarray(self.src_rate, dtype=np.float64))
        return Q

    def fixed_cells(self, N):
        """(mask, values): the prescribed cells and their pressures; a cell
        listed more than once takes the last value listed."""
        mask = np.zeros(N, bool)
        val = np.zeros(N)
        for c, v in zip(np.asarray(self.fix_cell, np.int64).tolist(),
                        np.asarray(self.fix_value, np.float64).tolist()):
            mask[c] = True
            val[c] = v
        return mask, val


@dataclass(frozen=True)
class Faces:
    """Internal faces (lo, hi, T) and Dirichlet faces (cell, T, p_b)."""
    lo: np.ndarray
    hi: np.ndarray
    T: np.ndarray
    b_cell: np.ndarray
    b_T: np.ndarray
    b_p: np.ndarray


def transmissibilities(g: Grid, kx, ky, kz, mu: float, bc: BC) -> Faces:
    """TPFA transmissibilities (Reading R2).

    Internal face between cells a and b along direction d with spacing h_d
    and face area A_d:  T = A_d / (h_d/(2 lambda_a) + h_d/(2 lambda_b)).
    Dirichlet face of cell a:  T_b = A_d / (h_d/(2 lambda_a)).
    """
    x, y, z = g.coords()
    i = np.arange(g.N)
    lam = [np.asarray(kx, float) / mu, np.asarray(ky, float) / mu, np.asarray(kz, float) / mu]
    h = [g.dx, g.dy, g.dz]
    area = [g.dy * g.dz, g.dx * g.dz, g.dx * g.dy]
    stride = [1, g.nx, g.nx * g.ny]
    coord = [x, y, z]
    n = [g.nx, g.ny, g.nz]
    lo_l, hi_l, T_l = [], [], []
    for d in range(3):
        a = i[coord[d] < n[d] - 1]
        b = a + stride[d]
        T = area[d] / (h[d] / (2.0 * lam[d][a]) + h[d] / (2.0 * lam[d][b]))
        lo_l.append(a); hi_l.append(b); T_l.append(T)
    lo = np.concatenate(lo_l); hi = np.concatenate(hi_l); T = np.concatenate(T_l)
    if bc.dirichlet:
        west = i[x == 0]
        east = i[x == g.nx - 1]
        cells = np.concatenate([west, east])
        Tb = area[0] / (h[0] / (2.0 * lam[0][cells]))
        pb = np.concatenate([np.full(west.size, bc.p_west), np.full(east.size, bc.p_east)])
    else:
        cells = np.zeros(0, np.int64); Tb = np.zeros(0); pb = np.zeros(0)
    return Faces(lo, hi, T, cells, Tb, pb)


@dataclass(frozen=True)
class Problem:
    grid: Grid
    fluid: Fluid
    bc: BC
    faces: Faces
    Q: np.ndarray     # integrated volumetric source per cell
    fixed: np.ndarray = None   # bool mask of the prescribed cells (Reading R19)
    p_fix: np.ndarray = None   # their pressures (0 elsewhere)

    @staticmethod
    def build(grid: Grid, fluid: Fluid, bc: BC, kx, ky, kz) -> "Problem":
        mask, val = bc.fixed_cells(grid.N)
        return Problem(grid, fluid, bc, transmissibilities(grid, kx, ky, kz, fluid.mu, bc),
                       bc.source_vector(grid.N), mask, val)

    @property
    def has_fixed(self) -> bool:
        return self.fixed is not None and bool(self.fixed.any())

    def with_fixed(self, p):
        """A copy of p carrying the prescribed values at the fixed cells."""
        p = np.array(p, dtype=np.float64, copy=True)
        if self.has_fixed:
            p[self.fixed] = self.p_fix[self.fixed]
        return p


def eliminate_fixed(M: sp.csr_matrix, fixed: np.ndarray) -> sp.csr_matrix:
    """Symmetric elimination of the fixed unknowns (Reading R19): every entry
    in a row or a column of a fixed cell is dropped, then each fixed row gets
    a unit diagonal."""
    coo = M.tocoo()
    keep = ~(fixed[coo.row] | fixed[coo.col])
    F = np.flatnonzero(fixed)
    rows = np.concatenate([coo.row[keep], F])
    cols = np.concatenate([coo.col[keep], F])
    vals = np.concatenate([coo.data[keep], np.ones(F.size)])
    out = sp.coo_matrix((vals, (rows, cols)), shape=M.shape).tocsr()
    out.sum_duplicates()
    out.sort_indices()
    return out


def _flux_sum(pb: Problem, rho, p):
    """Sum over the faces of cell i of the mass flux leaving i:
    sum_j T rho_f (p_i - p_j) + sum_b T_b rho_b (p_i - p_b)."""
    fc = pb.faces
    rho_f = 0.5 * (rho[fc.lo] + rho[fc.hi])                 # Reading R4
    q = fc.T * rho_f * (p[fc.lo] - p[fc.hi])
    out = np.zeros(pb.grid.N)
    np.add.at(out, fc.lo, q)
    np.add.at(out, fc.hi, -q)
    if fc.b_cell.size:
        rho_b = pb.fluid.rho(fc.b_p)
        np.add.at(out, fc.b_cell, fc.b_T * rho_b * (p[fc.b_cell] - fc.b_p))
    return out


def residual(pb: Problem, p, p_n, dt):
    """Discrete mass balance of Eq. 1 integrated over cell i and Eq. 2's
    implicit Euler step, in mass units (Reading R7 scaling):
    F_i = V phi (rho_i - rho_i^n)/dt + (fluxes leaving i) - rho_i Q_i."""
    fl = pb.fluid
    rho = fl.rho(p)
    rho_n = fl.rho(p_n)
    return (pb.grid.V * fl.phi * (rho - rho_n) / dt + _flux_sum(pb, rho, p)
            - rho * pb.Q)


def epsilon(pb: Problem, p, p_n, dt):
    """Nonlinear error of Eq. 19 per cell, with phi constant and S^n = 1:
    eps = q - phi/dt + (phi/dt) rho^n/rho + (1/rho) div(rho lambda grad p),
    where the cell-averaged divergence is minus the flux leaving the cell
    divided by V."""
    g, fl = pb.grid, pb.fluid
    rho = fl.rho(p)
    rho_n = fl.rho(p_n)
    q = pb.Q / g.V
    div = -_flux_sum(pb, rho, p) / g.V
    e = q - fl.phi / dt + (fl.phi / dt) * rho_n / rho + div / rho
    if pb.has_fixed:
        e[pb.fixed] = 0.0       # Reading R19: no equation at a fixed cell
    return e


@dataclass
class Linearised:
    A: sp.csr_matrix      # C + A~ (Eq. 6), rows scaled by V rho^nu
    f: np.ndarray         # b + C p^nu (Eq. 6), same scaling
    eps: np.ndarray       # Eq. 19 at p^nu
    rho: np.ndarray
    c: np.ndarray         # Eq. 4 at p^nu
    Cdiag: np.ndarray     # V rho c (the diagonal of C after scaling)


def accumulation_coefficient(fl: Fluid, p, p_n, dt):
    """Eq. 4 with d phi/dp = 0: c = (1/dt) [ - phi^n d(1/rho)/dp rho^n ]
    = phi rho^n rho'(p) / (dt rho(p)^2)."""
    rho = fl.rho(p)
    return fl.phi * fl.rho(p_n) * fl.drho(p) / (dt * rho * rho)


def flux_density_terms(pb: Problem, p, rho):
    """What the lagged step of Eq. 3 leaves out of the derivative of the
    paper's equation (Eq. 2 over rho, rows times V rho^nu; Reading R22):
    with Phi_i the mass flux leaving cell i and G_i = ... + Phi_i / (V rho_i),
      V rho_i dG_i/dp_j - (lagged row) = dPhi_i/dp_j|_(through rho_f)
                                         - delta_ij Phi_i rho'_i / rho_i.
    On a face (a, b) with q = T rho_f (p_a - p_b) and rho_f = (rho_a + rho_b)/2,
    q changes with p_a through rho_f by T rho'_a (p_a - p_b) / 2 (and alike
    for p_b); row a carries +q and row b carries -q.  The Dirichlet faces'
    density is fixed by the boundary value, so they add nothing there."""
    fl, fc = pb.fluid, pb.faces
    N = pb.grid.N
    dr = fl.drho(p)
    s = 0.5 * fc.T * (p[fc.lo] - p[fc.hi])
    phi_rho = _flux_sum(pb, rho, p) * dr / rho
    rows = np.concatenate([fc.lo, fc.lo, fc.hi, fc.hi, np.arange(N)])
    cols = np.concatenate([fc.lo, fc.hi, fc.lo, fc.hi, np.arange(N)])
    vals = np.concatenate([s * dr[fc.lo], s * dr[fc.hi], -s * dr[fc.lo], -s * dr[fc.hi], -phi_rho])
    X = sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()
    X.sum_duplicates()
    X.sort_indices()
    return X


def assemble(pb: Problem, p, p_n, dt, full_jacobian=False) -> Linearised:
    """Linear-system population (Table 1, step 1).

    Eq. 3 multiplied by V rho^nu gives, for the unknown p^{nu+1},
      V rho c (p^{nu+1} - p^nu) + sum_j T rho_f (p_i - p_j)^{nu+1}
          + sum_b T_b rho_b (p_i^{nu+1} - p_b) = V rho b
    with b from Eq. 5.  Hence A = C + A~ with C = diag(V rho c) and
    A~ the rho_f-weighted TPFA matrix including the Dirichlet faces, and
    f = V rho b + sum_b T_b rho_b p_b + C p^nu.
    full_jacobian adds the flux-density derivative terms of Reading R22
    (A is then not symmetric).
    """
    g, fl, fc = pb.grid, pb.fluid, pb.faces
    N, V = g.N, g.V
    p = pb.with_fixed(p)
    rho = fl.rho(p)
    rho_n = fl.rho(p_n)
    c = accumulation_coefficient(fl, p, p_n, dt)
    Cdiag = V * rho * c
    # Eq. 5 with phi constant: b = -phi/dt + phi rho^n/(dt rho) + q
    b = -fl.phi / dt + fl.phi * rho_n / (dt * rho) + pb.Q / V
    rho_f = 0.5 * (rho[fc.lo] + rho[fc.hi])
    w = fc.T * rho_f
    rows = [fc.lo, fc.hi, fc.lo, fc.hi]
    cols = [fc.lo, fc.hi, fc.hi, fc.lo]
    vals = [w, w, -w, -w]
    rhs_b = np.zeros(N)
    if fc.b_cell.size:
        wb = fc.b_T * fl.rho(fc.b_p)
        rows.append(fc.b_cell); cols.append(fc.b_cell); vals.append(wb)
        np.add.at(rhs_b, fc.b_cell, wb * fc.b_p)
    rows.append(np.arange(N)); cols.append(np.arange(N)); vals.append(Cdiag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    f = V * rho * b + rhs_b + Cdiag * p
    if full_jacobian:
        # Reading R22: A p^{nu+1} = f still means A dp = -F(p^nu), so the
        # added derivative terms X enter f as X p^nu.
        X = flux_density_terms(pb, p, rho)
        A = (A + X).tocsr()
        A.sum_duplicates()
        A.sort_indices()
        f = f + X @ p
    if pb.has_fixed:
        # Reading R19: with p_F known, row j of A p = f reads
        # sum_{k free} a_jk p_k = f_j - sum_{k fixed} a_jk p_k
        Fm = pb.fixed
        f = f - A[:, Fm] @ p[Fm]
        f[Fm] = p[Fm]
        A = eliminate_fixed(A, Fm)
    return Linearised(A, f, epsilon(pb, p, p_n, dt), rho, c, Cdiag)
