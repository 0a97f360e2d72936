"""The C-AMS procedure (Table 1) inside the Newton loop with linear-system
update adaptivity (Sec. 4.1.1) and adaptive operator updates (Sec. 4.1.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

One C-AMS iteration (Table 1 without correction functions, Sec. 4.1.4):
  (optional) n_pre ILU(0) steps   p <- p + M^{-1}(f - A p)
  multiscale stage (Eq. 15)       p <- p + P (R A P)^{-1} R (f - A p)
  post-smoothing, n_post times    p <- p + M^{-1}(f - A p)
Reading R11: the paper's only pre-smoother is the correction function, which
it drops; ILU(0) pre-smoothing is an option that defaults to 0 steps.  The
accumulated post-smoothing corrections form dp'^{nu+1} of Table 1, step 7.

Control (Sec. 4.1.1, Table 3):
  outer loop: assemble A, f, eps at p^nu; stop when ||eps||_2 < tol, then
  refactor ILU(0), update the basis adaptively, rebuild and factor R A P;
  inner loop: C-AMS iterations until ||r^i||_2 / ||r^0||_2 < 0.1.
Reading R13: the paper's stopping test is absolute (||eps||_2 < 1e-6); here
it is relative to ||eps|| at the start of the time step (p = p^n), and the
absolute form is available with tol_abs.
Reading R14: when the inner loop reaches its cap the outer loop still
re-linearises; hitting max_newton reports non-convergence.

Adaptive operator update (Sec. 4.1.2), Reading R15: the paper says the
changes of the entries of A and f are monitored.  Here every entity (edge
segment, face patch, dual-block interior) keeps a snapshot of the rows of its
basis operator A_b from its last build, and is rebuilt when the largest
relative change of those entries exceeds theta, or when an entity whose basis
values enter its right-hand side (a neighbouring entity one level lower) was
rebuilt in the same pass.  theta < 0 rebuilds everything every time.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .problem import Problem, assemble
from .wirebasket import Wirebasket, build_wirebasket
from .basis import basis_operator, correction_function, prolongation, PRows
from .coarse import restriction, coarse_operator, coarse_factor, coarse_solve
from .ilu import ilu0, ilu_apply


@dataclass
class Options:
    coarse: tuple = (5, 5, 1)
    basis: int = 4
    restriction: int = 0   # 0 MSFE, 1 MSFV, 2 MSFE then one closing MSFV correction (Sec. 4.3)
    n_pre: int = 0
    n_post: int = 1
    lin_rtol: float = 0.1
    nl_tol: float = 1e-6
    tol_abs: bool = False
    adapt_theta: float = 0.1
    max_newton: int = 50
    max_cams: int = 200
    cf: bool = False       # correction functions as the pre-smoother (Table 1 step 4, Reading R21)
    full_jacobian: bool = False   # Newton with the flux density differentiated (Reading R22)


class BasisState:
    """Prolongation operator plus the per-entity snapshots of Sec. 4.1.2."""

    def __init__(self, wb: Wirebasket):
        self.wb = wb
        self.P = PRows(wb.grid.N)
        self.snap = None           # A_b data array of the last build, per entity rows
        self.built = False
        self._deps = None

    def _dependencies(self, Ab):
        """For each entity, the entities one level lower that touch it."""
        wb = self.wb
        coo = Ab.tocoo()
        r, c = coo.row, coo.col
        er, ec = wb.entity[r], wb.entity[c]
        m = (er >= 0) & (ec >= 0) & (wb.level[c] == wb.level[r] - 1)
        deps = [set() for _ in wb.entities]
        for a, b in zip(er[m].tolist(), ec[m].tolist()):
            deps[a].add(b)
        return deps

    def update(self, Ab, theta: float, force=False) -> int:
        """Rebuild the flagged entities; returns how many were rebuilt."""
        wb = self.wb
        ne = len(wb.entities)
        if self._deps is None:
            self._deps = self._dependencies(Ab)
        if not self.built or force or theta < 0:
            flag = np.ones(ne, bool)
        else:
            rowcell = np.repeat(np.arange(Ab.shape[0]), np.diff(Ab.indptr))
            a, s = Ab.data, self.snap
            nz = s != 0.0
            rel = np.zeros_like(a)
            rel[nz] = np.abs(a[nz] - s[nz]) / np.abs(s[nz])
            rel[(~nz) & (a != 0.0)] = np.inf
            per_cell = np.zeros(Ab.shape[0])
            np.maximum.at(per_cell, rowcell, rel)
            flag = np.zeros(ne, bool)
            ent = wb.entity
            m = ent >= 0
            per_ent = np.zeros(ne)
            np.maximum.at(per_ent, ent[m], per_cell[m])
            flag = per_ent > theta
            # dependency propagation, lower levels first
            for k in range(2, wb.d_active + 1):
                for ei, e in enumerate(wb.entities):
                    if e.level == k and not flag[ei]:
                        if any(flag[d] for d in self._deps[ei]):
                            flag[ei] = True
        prolongation(Ab, wb, self.P, rebuild=flag)
        if self.snap is None:
            self.snap = Ab.data.copy()
        else:
            rowcell = np.repeat(np.arange(Ab.shape[0]), np.diff(Ab.indptr))
            ent_of_entry = wb.entity[rowcell]
            upd = (ent_of_entry >= 0) & flag[np.maximum(ent_of_entry, 0)]
            self.snap[upd] = Ab.data[upd]
        self.built = True
        return int(flag.sum())

    def matrix(self):
        return self.P.to_csr(self.wb.Nc)


def cams_iteration(A, f, p, P, R, lu, LU, n_pre, n_post, cf=None):
    """One C-AMS iteration (Table 1, steps 4-7, ILU(0) smoother); cf, when
    given, maps a residual to its correction function (the pre-smoothing
    stage of step 4)."""
    if cf is not None:
        p = p + cf(f - A @ p)
    for _ in range(n_pre):
        p = p + ilu_apply(LU, f - A @ p)
    r = f - A @ p
    p = p + P @ coarse_solve(lu, R @ r)          # Eq. 15
    for _ in range(n_post):
        p = p + ilu_apply(LU, f - A @ p)
    return p


@dataclass
class StepStats:
    newton_its: int = 0
    cams_its: int = 0
    basis_rebuilt: int = 0
    converged: bool = False
    eps_hist: list = field(default_factory=list)
    cams_per_newton: list = field(default_factory=list)
    res_final: float = 0.0
    msfv_final: bool = False     # the closing MSFV correction was applied (restriction 2)


def solve_step(pb: Problem, wb: Wirebasket, state: BasisState, opt: Options,
               p_n: np.ndarray, dt: float, p_init=None):
    """One implicit time step from p^n: returns (p^{n+1}, StepStats)."""
    check_fixed(pb, wb)
    p = pb.with_fixed(p_n if p_init is None else p_init)
    st = StepStats()
    eps0 = None
    for nu in range(opt.max_newton + 1):
        lin = assemble(pb, p, p_n, dt, opt.full_jacobian)
        en = float(np.linalg.norm(lin.eps))
        st.eps_hist.append(en)
        if eps0 is None:
            eps0 = en
        ref = 1.0 if opt.tol_abs else eps0
        if en == 0.0 or en < opt.nl_tol * ref:
            st.converged = True
            break
        if nu == opt.max_newton:
            break
        LU = ilu0(lin.A)
        Ab = basis_operator(pb, opt.basis, lin.rho, lin.c, p_n, dt)
        st.basis_rebuilt += state.update(Ab, opt.adapt_theta)
        P = state.matrix()
        R = restriction(0 if opt.restriction == 2 else opt.restriction, P, wb)
        lu = coarse_factor(coarse_operator(R, lin.A, P))
        r0 = float(np.linalg.norm(lin.f - lin.A @ p))
        its = 0
        while its < opt.max_cams:
            cf = (lambda r: correction_function(Ab, wb, r)) if opt.cf else None
            p = cams_iteration(lin.A, lin.f, p, P, R, lu, LU, opt.n_pre, opt.n_post, cf)
            its += 1
            rn = float(np.linalg.norm(lin.f - lin.A @ p))
            if rn < opt.lin_rtol * r0:
                break
        st.res_final = rn
        st.cams_its += its
        st.cams_per_newton.append(its)
        st.newton_its += 1
    if opt.restriction == 2 and st.converged and st.newton_its > 0:
        # Sec. 4.3: converge with MSFE, then one MSFV coarse correction of the
        # last linearisation (A, f at the converged p) with the current basis:
        # p <- p + P (R_FV A P)^{-1} R_FV (f - A p).  Afterwards R_FV (f - A p)
        # vanishes: the linearised fluxes balance on every primal block.
        P = state.matrix()
        Rfv = restriction(1, P, wb)
        lu_fv = coarse_factor(coarse_operator(Rfv, lin.A, P))
        p = p + P @ coarse_solve(lu_fv, Rfv @ (lin.f - lin.A @ p))
        st.msfv_final = True
    return p, st


def check_fixed(pb: Problem, wb: Wirebasket):
    """Reading R19: a prescribed-pressure cell may not be a coarse node."""
    if pb.has_fixed and np.any(wb.level[pb.fixed] == 0):
        raise ValueError("a fixed cell is a coarse node")


def run(pb: Problem, opt: Options, p0: np.ndarray, dt, steps: int):
    """Several implicit steps of size dt (a number, or one per step);
    returns (p, [StepStats per step])."""
    wb = build_wirebasket(pb.grid, opt.coarse)
    state = BasisState(wb)
    dts = [float(dt)] * steps if np.ndim(dt) == 0 else [float(v) for v in dt][:steps]
    p = p0.copy()
    stats = []
    for d in dts:
        p, st = solve_step(pb, wb, state, opt, p, d)
        stats.append(st)
    return p, stats
