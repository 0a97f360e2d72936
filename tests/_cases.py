"""Shared construction of one case for both sides: the oracle problem and
the GPU handle receive the same seeded arrays from workloads/."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle
from workloads import WORKLOADS, make_inputs


@dataclass
class Case:
    w: object
    inp: dict
    pb: object
    opt: object        # oracle.Options

    @property
    def N(self):
        return self.w.nx * self.w.ny * self.w.nz


def make_case(name=None, w=None, seed=0, **overrides):
    if w is None:
        w = WORKLOADS[name]
    if overrides:
        w = w.with_(**overrides)
    inp = make_inputs(w, seed)
    g = oracle.Grid(w.nx, w.ny, w.nz, inp["dx"], inp["dy"], inp["dz"])
    fl = oracle.Fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi)
    bc = oracle.BC(inp["dirichlet"], w.p_west, w.p_east, inp["src_cell"], inp["src_rate"],
                   inp["fix_cell"], inp["fix_value"])
    pb = oracle.Problem.build(g, fl, bc, inp["kx"], inp["ky"], inp["kz"])
    opt = oracle.Options(coarse=w.coarse, basis=w.basis, restriction=w.restriction,
                         n_pre=w.n_pre, n_post=w.n_post, lin_rtol=w.lin_rtol, nl_tol=w.nl_tol,
                         adapt_theta=w.adapt_theta, max_newton=w.max_newton,
                         max_cams=w.max_cams)
    return Case(w, inp, pb, opt)


def gpu_handle(case: Case, memspace=0, **extra):
    """A library handle for the case; extra options (e.g. cf=True) go to
    make_options."""
    from paper_1705_05783_gb300 import cams
    w, inp = case.w, case.inp
    grid = cams.cams_grid(w.nx, w.ny, w.nz, inp["dx"], inp["dy"], inp["dz"])
    fluid = cams.cams_fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi)
    opt = cams.make_options(w.coarse, basis=w.basis, restriction=w.restriction, n_pre=w.n_pre,
                            n_post=w.n_post, lin_rtol=w.lin_rtol, nl_tol=w.nl_tol,
                            adapt_theta=w.adapt_theta, max_newton=w.max_newton,
                            max_cams=w.max_cams, memspace=memspace, precision=w.precision,
                            **extra)
    h = cams.cams_setup(grid, fluid, opt, inp["kx"], inp["ky"], inp["kz"])
    bc, keep = cams.make_bc(inp["dirichlet"], w.p_west, w.p_east,
                            inp["src_cell"] if len(inp["src_cell"]) else None,
                            inp["src_rate"] if len(inp["src_rate"]) else None,
                            inp["fix_cell"] if len(inp["fix_cell"]) else None,
                            inp["fix_value"] if len(inp["fix_value"]) else None)
    return h, bc, keep


def p_from_gpu(h, N, Nc):
    """P as a scipy CSR matrix from the ELL-8 slots."""
    import scipy.sparse as sp
    from paper_1705_05783_gb300 import cams
    vals = cams.cams_get(h, cams.CAMS_Q_PROLONG, np.zeros(8 * N))
    cols = cams.cams_get_int(h, cams.CAMS_Q_PROLONG_J, np.zeros(8 * N, np.int32))
    rows = np.tile(np.arange(N), 8)
    m = cols >= 0
    return sp.csr_matrix((vals[m], (rows[m], cols[m])), shape=(N, Nc)), vals, cols


def coarse_from_gpu(h, nc):
    """27-point coarse stencil -> dense matrix in the natural coarse order."""
    from paper_1705_05783_gb300 import cams
    Nc = nc[0] * nc[1] * nc[2]
    st = cams.cams_get(h, cams.CAMS_Q_COARSE, np.zeros(27 * Nc))
    A = np.zeros((Nc, Nc))
    for I in range(Nc):
        Ic = (I % nc[0], (I // nc[0]) % nc[1], I // (nc[0] * nc[1]))
        for t in range(27):
            off = (t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1)
            J = [Ic[d] + off[d] for d in range(3)]
            if all(0 <= J[d] < nc[d] for d in range(3)):
                A[I, J[0] + nc[0] * (J[1] + nc[1] * J[2])] = st[27 * I + t]
    return A, st


def matrix_from_gpu(h, N):
    from paper_1705_05783_gb300 import cams
    m = cams.cams_get(h, cams.CAMS_Q_MATRIX, np.zeros(4 * N))
    return m[:N], m[N:2 * N], m[2 * N:3 * N], m[3 * N:]
