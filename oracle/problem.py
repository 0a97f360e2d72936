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
    Q_i = q_i dV_i (the integrated source of Eq. 6), positive = injection."""
    dirichlet: bool = True
    p_west: float = 1.0
    p_east: float = 0.0
    src_cell: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    src_rate: np.ndarray = field(default_factory=lambda: np.zeros(0))

    def source_vector(self, N):
        Q = np.zeros(N)
        np.add.at(Q, np.asarray(self.src_cell, dtype=np.int64), np.asarray(self.src_rate, dtype=np.float64))
        return Q


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

    @staticmethod
    def build(grid: Grid, fluid: Fluid, bc: BC, kx, ky, kz) -> "Problem":
        return Problem(grid, fluid, bc, transmissibilities(grid, kx, ky, kz, fluid.mu, bc),
                       bc.source_vector(grid.N))


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
    return q - fl.phi / dt + (fl.phi / dt) * rho_n / rho + div / rho


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


def assemble(pb: Problem, p, p_n, dt) -> Linearised:
    """Linear-system population (Table 1, step 1).

    Eq. 3 multiplied by V rho^nu gives, for the unknown p^{nu+1},
      V rho c (p^{nu+1} - p^nu) + sum_j T rho_f (p_i - p_j)^{nu+1}
          + sum_b T_b rho_b (p_i^{nu+1} - p_b) = V rho b
    with b from Eq. 5.  Hence A = C + A~ with C = diag(V rho c) and
    A~ the rho_f-weighted TPFA matrix including the Dirichlet faces, and
    f = V rho b + sum_b T_b rho_b p_b + C p^nu.
    """
    g, fl, fc = pb.grid, pb.fluid, pb.faces
    N, V = g.N, g.V
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
    return Linearised(A, f, epsilon(pb, p, p_n, dt), rho, c, Cdiag)
