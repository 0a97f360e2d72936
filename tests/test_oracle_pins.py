"""Pins of the CPU oracle against facts fixed by the paper and by the
mathematics: closed forms, invariants, textbook special cases, brute force.
None of these tests re-types an oracle formula; each would fail on a
plausible mistake (sign, index, dropped term, transposed operand)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import (BC, Fluid, Grid, Options, Problem, assemble, basis_operator,
                    build_wirebasket, cams_iteration, coarse_operator, ilu0, ilu_apply,
                    prolongation, prolongation_global, restriction, run)
from oracle.basis import PRows
from oracle.coarse import coarse_factor, coarse_solve
from oracle.problem import accumulation_coefficient, residual, epsilon
from oracle.solver import BasisState, solve_step

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(nx, ny, nz):
    h = 1.0 / nx
    return Grid(nx, ny, nz, h, h, h)


def _lognormal(N, rng, s=1.5):
    k = np.exp(s * rng.standard_normal(N))
    return k, k.copy(), k.copy()


def _problem(g, k, law=0, c=0.1, dirichlet=True, src=None):
    fl = Fluid(law, c, 1.0, 1.0, 0.1)
    bc = BC(dirichlet, 1.0, 0.0) if src is None else BC(dirichlet, 1.0, 0.0, *src)
    return Problem.build(g, fl, bc, *k)


# ---------------------------------------------------------------- Sec. 2 --

def test_tpfa_series_resistance(rng):
    """1D incompressible steady flow through layers: the flux equals
    Delta p / sum_i (h / (A k_i)) (resistances in series) on every face."""
    n = 17
    g = Grid(n, 1, 1, 0.3, 2.0, 0.5)
    k = np.exp(2.0 * rng.standard_normal(n))
    pb = _problem(g, (k, k, k), law=1, c=0.0)        # rho = 1: incompressible
    lin = assemble(pb, np.zeros(n), np.zeros(n), 1.0)
    p = spl.spsolve(lin.A.tocsc(), lin.f)
    area = g.dy * g.dz
    q_exact = (1.0 - 0.0) / np.sum(g.dx / (area * k))
    fc = pb.faces
    q = fc.T * (p[fc.lo] - p[fc.hi])
    np.testing.assert_allclose(q, q_exact, rtol=1e-12)


@pytest.mark.parametrize("shape,coarse", [((12, 1, 1), (4, 1, 1)), ((10, 10, 1), (5, 5, 1)),
                                          ((8, 6, 4), (4, 3, 2))])
def test_linear_pressure_closed_form(shape, coarse):
    """Homogeneous k, incompressible, Dirichlet 1/0 on west/east: TPFA
    reproduces p_i = 1 - (x_i + 1/2)/nx exactly, and C-AMS converges to it."""
    g = _grid(*shape)
    one = np.ones(g.N)
    pb = _problem(g, (one, one, one), law=1, c=0.0)
    opt = Options(coarse=coarse, basis=4, n_post=2, nl_tol=1e-13, max_newton=20)
    p, st = run(pb, opt, np.zeros(g.N), 1e-3, 1)
    x, _, _ = g.coords()
    np.testing.assert_allclose(p, 1.0 - (x + 0.5) / g.nx, atol=1e-12)
    assert st[0].converged


def test_epsilon_matches_linear_residual(rng):
    """Eq. 19 and Eqs. 3-6 are two statements of one balance: at p^nu,
    f - A p^nu = V rho eps = -F(p^nu)."""
    g = _grid(6, 5, 4)
    k = _lognormal(g.N, rng)
    src = (np.array([3, 50]), np.array([0.7, -0.4]))
    for law, c in ((0, 0.3), (1, 0.8)):
        pb = _problem(g, k, law=law, c=c, src=src)
        p = rng.uniform(-0.5, 1.5, g.N)
        pn = rng.uniform(-0.5, 1.5, g.N)
        lin = assemble(pb, p, pn, 0.01)
        r = lin.f - lin.A @ p
        np.testing.assert_allclose(r, g.V * lin.rho * lin.eps, rtol=1e-10, atol=1e-12 * np.abs(r).max())
        np.testing.assert_allclose(r, -residual(pb, p, pn, 0.01), rtol=1e-10, atol=1e-12 * np.abs(r).max())


@pytest.mark.parametrize("law,c", [(0, 0.2), (1, 1.0)])
def test_accumulation_coefficient_is_derivative(law, c):
    """Eq. 4: c = d/dp [ phi/dt - phi rho^n / (dt rho(p)) ] (complex step)."""
    fl = Fluid(law, c, 1.3, 1.0, 0.1)
    p = np.linspace(-0.4, 1.2, 9)
    pn = np.linspace(0.3, -0.2, 9)
    dt = 0.02
    hstep = 1e-30
    pz = p + 1j * hstep
    rho_z = fl.rho0 * (np.exp(c * pz) if law == 0 else (1 + c * pz))
    g = -fl.phi * fl.rho(pn) / (dt * rho_z)
    np.testing.assert_allclose(accumulation_coefficient(fl, p, pn, dt), g.imag / hstep, rtol=1e-13)


def test_global_mass_balance(rng):
    """Internal fluxes cancel: sum_i F_i = accumulation + Dirichlet boundary
    flux - sources, for any p."""
    g = _grid(7, 5, 3)
    k = _lognormal(g.N, rng)
    src = (np.array([0, 100]), np.array([0.5, -0.25]))
    pb = _problem(g, k, c=0.4, src=src)
    p = rng.uniform(0, 1, g.N)
    pn = rng.uniform(0, 1, g.N)
    F = residual(pb, p, pn, 0.05)
    fl, fc = pb.fluid, pb.faces
    acc = g.V * fl.phi * np.sum(fl.rho(p) - fl.rho(pn)) / 0.05
    bnd = np.sum(fc.b_T * fl.rho(fc.b_p) * (p[fc.b_cell] - fc.b_p))
    srcs = np.sum(fl.rho(p)[src[0]] * src[1])
    assert abs(F.sum() - (acc + bnd - srcs)) < 1e-11 * (abs(acc) + abs(bnd) + 1)


def test_flux_divergence_second_order():
    """Consistency with Eq. 1: for homogeneous k and a smooth pressure the
    cell-averaged flux divergence of Eq. 19 tends to div(rho lambda grad p)
    at second order in h."""
    def err(n):
        g = Grid(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n)
        one = np.ones(g.N)
        fl = Fluid(0, 0.5, 1.0, 1.0, 0.1)
        pb = Problem.build(g, fl, BC(False), one, one, one)
        x, y, z = [(c + 0.5) / n for c in g.coords()]
        P = lambda x, y, z: np.sin(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        p = P(x, y, z)
        # interior cells only (the no-flow boundary is not consistent with P)
        inner = (g.coords()[0] > 0) & (g.coords()[0] < n - 1) & (g.coords()[1] > 0) & \
                (g.coords()[1] < n - 1) & (g.coords()[2] > 0) & (g.coords()[2] < n - 1)
        dt = 1.0
        eps = epsilon(pb, p, p, dt)          # accumulation cancels with p_n = p
        rho = fl.rho(p)
        num = eps * rho                      # = div(rho lambda grad p), q = 0
        # exact: div(exp(c p) grad p) = exp(c p) (c |grad p|^2 + lap p)
        c, pi = 0.5, np.pi
        px = pi * np.cos(pi * x) * np.cos(pi * y) * np.cos(pi * z)
        py = -pi * np.sin(pi * x) * np.sin(pi * y) * np.cos(pi * z)
        pz = -pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z)
        lap = -3 * pi ** 2 * p
        exact = np.exp(c * p) * (c * (px ** 2 + py ** 2 + pz ** 2) + lap)
        return np.max(np.abs(num - exact)[inner])
    e1, e2 = err(24), err(48)
    assert 3.4 < e1 / e2 < 4.6


def test_dense_direct_newton(rng):
    """O-exact: the C-AMS solution is the root of the nonlinear residual, as
    found by a plain Newton iteration with a finite-difference Jacobian and
    dense LU (tiny grid, compressible, heterogeneous, wells)."""
    g = _grid(6, 6, 4)
    k = _lognormal(g.N, rng, 1.0)
    src = (np.array([0, g.N - 1]), np.array([0.02, -0.02]))
    for dirichlet in (True, False):
        pb = _problem(g, k, c=0.5, dirichlet=dirichlet, src=src)
        pn = np.zeros(g.N)
        dt = 0.005
        p = pn.copy()
        for _ in range(30):
            F = residual(pb, p, pn, dt)
            J = np.zeros((g.N, g.N))
            for j in range(g.N):
                e = np.zeros(g.N); e[j] = 1e-7
                J[:, j] = (residual(pb, p + e, pn, dt) - residual(pb, p - e, pn, dt)) / 2e-7
            p = p - np.linalg.solve(J, F)
            if np.linalg.norm(F) < 1e-15:
                break
        for R in (0, 1):
            opt = Options(coarse=(3, 3, 2), basis=4, restriction=R, n_post=3, nl_tol=1e-12)
            q, st = run(pb, opt, pn, dt, 1)
            assert st[0].converged
            np.testing.assert_allclose(q, p, rtol=0, atol=1e-10 * np.abs(p).max())


# ---------------------------------------------------------------- Sec. 3 --

def test_wirebasket_golden_2d():
    rows = [l.strip() for l in open(os.path.join(GOLDEN, "wirebasket_10x10_b5x5.txt"))
            if l.strip() and not l.startswith("#")]
    want = np.array([[{"V": 0, "E": 1, "I": 2}[ch] for ch in r] for r in rows])
    wb = build_wirebasket(_grid(10, 10, 1), (5, 5, 1))
    np.testing.assert_array_equal(wb.level.reshape(10, 10), want)
    assert wb.Nc == 4


def test_wirebasket_counts_3d():
    """Level counts of a 6x6x4 grid with 3x3x2 blocks follow from the number
    of vertex coordinates per direction (2, 2, 2) and non-vertex ones (4, 4, 2)."""
    wb = build_wirebasket(_grid(6, 6, 4), (3, 3, 2))
    counts = np.bincount(wb.level, minlength=4)
    np.testing.assert_array_equal(counts, [8, 16 + 16 + 8, 32 + 16 + 16, 32])
    # every entity's corners are vertices; each non-vertex cell is in one entity
    assert np.all((wb.entity >= 0) == (wb.level > 0))
    assert sum(len(e.cells) for e in wb.entities) == np.count_nonzero(wb.level)


def _P(g, k, coarse, basis, pb=None, p=None):
    pb = pb or _problem(g, k)
    p = np.zeros(g.N) if p is None else p
    lin = assemble(pb, p, np.zeros(g.N), 0.01)
    Ab = basis_operator(pb, basis, lin.rho, lin.c, np.zeros(g.N), 0.01)
    wb = build_wirebasket(g, coarse)
    return prolongation(Ab, wb).to_csr(wb.Nc), wb, Ab, lin


@pytest.mark.parametrize("basis", [4, 2])
def test_partition_of_unity(rng, basis):
    g = _grid(12, 10, 6)
    P, wb, _, _ = _P(g, _lognormal(g.N, rng, 2.0), (4, 5, 3), basis,
                     p=None)
    s = np.asarray(P.sum(axis=1)).ravel()
    np.testing.assert_allclose(s, 1.0, atol=1e-13)
    assert P.data.min() >= -1e-14 and P.data.max() <= 1 + 1e-14


@pytest.mark.parametrize("basis", [1, 3])
def test_compressible_basis_not_unity(rng, basis):
    """Fig. 2: with the accumulation term the basis functions decay and do
    not sum to one (but stay non-negative)."""
    g = _grid(12, 10, 6)
    k = _lognormal(g.N, rng, 1.0)
    pb = _problem(g, k, c=2.0)
    P, wb, _, _ = _P(g, k, (4, 5, 3), basis, pb=pb, p=np.full(g.N, 0.3))
    s = np.asarray(P.sum(axis=1)).ravel()
    nv = wb.level > 0
    assert np.all(s[nv] < 1.0) and np.all(s[~nv] == 1.0)
    assert P.data.min() >= 0.0


def _hat(n, b, x):
    """1D basis values of every coarse node at fine coordinate x for
    homogeneous coefficients: linear between neighbouring nodes, constant
    beyond the first/last node."""
    nc = n // b
    v = np.arange(nc) * b + b // 2
    out = np.zeros(nc)
    if x <= v[0]:
        out[0] = 1.0
    elif x >= v[-1]:
        out[-1] = 1.0
    else:
        J = np.searchsorted(v, x, side="right") - 1
        t = (x - v[J]) / b
        out[J] = 1 - t
        out[J + 1] = t
    return out


@pytest.mark.parametrize("shape,coarse", [((15, 1, 1), (5, 1, 1)), ((12, 8, 1), (4, 4, 1)),
                                          ((8, 9, 6), (4, 3, 3))])
def test_homogeneous_basis_is_multilinear(shape, coarse):
    """For homogeneous k and (B4) the reduced-problem basis functions are the
    tensor products of 1D linear hats (bilinear/trilinear are discrete
    harmonic for the 5-/7-point stencil)."""
    g = _grid(*shape)
    one = np.ones(g.N)
    P, wb, _, _ = _P(g, (one, one, one), coarse, 4)
    P = P.toarray()
    x, y, z = g.coords()
    for i in range(g.N):
        hx = _hat(g.nx, coarse[0], x[i]) if g.nx > 1 else np.ones(1)
        hy = _hat(g.ny, coarse[1], y[i]) if g.ny > 1 else np.ones(1)
        hz = _hat(g.nz, coarse[2], z[i]) if g.nz > 1 else np.ones(1)
        want = np.einsum("k,j,i->kji", hz, hy, hx).ravel()
        np.testing.assert_allclose(P[i], want, atol=1e-13)


@pytest.mark.parametrize("basis", [1, 4])
def test_staged_basis_equals_global_reduced_solve(rng, basis):
    g = _grid(12, 10, 6)
    k = _lognormal(g.N, rng, 2.0)
    pb = _problem(g, k, c=1.0)
    P, wb, Ab, _ = _P(g, k, (4, 5, 3), basis, pb=pb, p=np.full(g.N, 0.2))
    Pg = prolongation_global(Ab, wb)
    np.testing.assert_allclose(P.toarray(), Pg.toarray(), atol=1e-12)


def test_msfe_coarse_matrix_symmetric_spd(rng):
    g = _grid(12, 10, 6)
    k = _lognormal(g.N, rng, 2.0)
    P, wb, _, lin = _P(g, k, (4, 5, 3), 4)
    Ac = coarse_operator(restriction(0, P, wb), lin.A, P)
    assert np.abs(Ac - Ac.T).max() <= 1e-14 * np.abs(Ac).max()
    np.linalg.cholesky(Ac)


@pytest.mark.parametrize("R", [0, 1])
def test_multiscale_stage_exact_on_coarse_space(rng, R):
    """If the solution lies in range(P), one multiscale stage (Eq. 14)
    recovers it from any start."""
    g = _grid(12, 10, 6)
    k = _lognormal(g.N, rng, 2.0)
    P, wb, _, lin = _P(g, k, (4, 5, 3), 4)
    Rm = restriction(R, P, wb)
    pc = rng.standard_normal(wb.Nc)
    pstar = P @ pc
    f = lin.A @ pstar
    lu = coarse_factor(coarse_operator(Rm, lin.A, P))
    LU = ilu0(lin.A)
    p = cams_iteration(lin.A, f, np.zeros(g.N), P, Rm, lu, LU, 0, 0)
    np.testing.assert_allclose(p, pstar, atol=1e-11 * np.abs(pstar).max())


def test_msfv_local_conservation(rng):
    """After an MSFV stage the restricted residual vanishes block by block
    (locally conservative, Sec. 4)."""
    g = _grid(12, 10, 6)
    k = _lognormal(g.N, rng, 2.0)
    P, wb, _, lin = _P(g, k, (4, 5, 3), 4)
    Rm = restriction(1, P, wb)
    lu = coarse_factor(coarse_operator(Rm, lin.A, P))
    p0 = rng.standard_normal(g.N)
    r = lin.f - lin.A @ p0
    p1 = p0 + P @ coarse_solve(lu, Rm @ r)
    blk = Rm @ (lin.f - lin.A @ p1)
    scale = np.abs(Rm @ np.abs(lin.f - lin.A @ p0)).max()
    assert np.abs(blk).max() <= 1e-12 * scale


def test_msfe_1d_homogeneous_coarse_laplacian():
    """1D homogeneous, incompressible, (B4) + MSFE: the Galerkin coarse matrix
    is the 3-point Laplacian of the coarse grid, coarse transmissibility
    T / b, on rows away from the boundary."""
    n, b = 30, 5
    g = Grid(n, 1, 1, 1.0, 1.0, 1.0)
    one = np.ones(n)
    pb = _problem(g, (one, one, one), law=1, c=0.0)
    P, wb, _, lin = _P(g, (one, one, one), (b, 1, 1), 4, pb=pb)
    Ac = coarse_operator(restriction(0, P, wb), lin.A, P)
    T = 1.0
    for J in range(1, wb.Nc - 1):
        np.testing.assert_allclose(Ac[J, J - 1:J + 2], [-T / b, 2 * T / b, -T / b], atol=1e-14)


def _dense_ilu_check(A, L, U):
    A = A.toarray(); LU = (L @ U).toarray()
    mask = A != 0
    np.testing.assert_allclose(LU[mask], A[mask], atol=1e-13 * np.abs(A).max())
    assert np.all(L.toarray()[np.triu_indices(A.shape[0], 1)] == 0)
    assert np.all(U.toarray()[np.tril_indices(A.shape[0], -1)] == 0)
    # the factors keep the pattern of A (no fill)
    Lm, Um = L.toarray(), U.toarray()
    off = ~mask & ~np.eye(A.shape[0], dtype=bool)
    assert np.all(Lm[off] == 0) and np.all(Um[off] == 0)


def test_ilu0_reproduces_A_on_its_pattern(rng):
    g = _grid(5, 4, 3)
    pb = _problem(g, _lognormal(g.N, rng), c=0.3)
    lin = assemble(pb, rng.uniform(0, 1, g.N), np.zeros(g.N), 0.02)
    L, U = ilu0(lin.A)
    _dense_ilu_check(lin.A, L, U)
    # a non-symmetric matrix with the same pattern
    B = lin.A.copy(); B.data = B.data * rng.uniform(0.5, 1.5, B.data.size)
    B = B + sp.diags(np.abs(B).sum(axis=1).A1)
    L, U = ilu0(B.tocsr())
    _dense_ilu_check(B.tocsr(), L, U)


def test_ilu0_tridiagonal_is_exact(rng):
    """No fill for a tridiagonal matrix: ILU(0) = LU and one smoothing step
    solves the 1D system."""
    g = Grid(20, 1, 1, 1.0, 1.0, 1.0)
    pb = _problem(g, _lognormal(20, rng), c=0.2)
    lin = assemble(pb, np.zeros(20), np.zeros(20), 0.1)
    LU = ilu0(lin.A)
    p = ilu_apply(LU, lin.f)
    np.testing.assert_allclose(lin.A @ p, lin.f, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p, sla.solve(lin.A.toarray(), lin.f), rtol=1e-12, atol=1e-15)


def test_ilu0_diagonal_recursion_7point(rng):
    """For a 7-point stencil in natural order ILU(0) only changes the
    diagonal: d_i = a_ii - sum_{j lower nbr} a_ij a_ji / d_j."""
    g = _grid(6, 5, 4)
    pb = _problem(g, _lognormal(g.N, rng), c=0.3)
    A = assemble(pb, rng.uniform(0, 1, g.N), np.zeros(g.N), 0.02).A.toarray()
    d = np.zeros(g.N)
    for i in range(g.N):
        d[i] = A[i, i]
        for j in (i - 1, i - g.nx, i - g.nx * g.ny):
            if j >= 0 and A[i, j] != 0:
                d[i] -= A[i, j] * A[j, i] / d[j]
    L, U = ilu0(sp.csr_matrix(A))
    np.testing.assert_allclose(U.diagonal(), d, rtol=1e-14)
    np.testing.assert_array_equal(sp.triu(U, 1).toarray(), np.triu(A, 1))


# ------------------------------------------------------- Sec. 4.1.1/4.1.2 --

def test_adaptive_basis_updates(rng):
    g = _grid(12, 10, 6)
    k = _lognormal(g.N, rng, 1.5)
    pb = _problem(g, k, c=1.0)
    wb = build_wirebasket(g, (4, 5, 3))
    ne = len(wb.entities)
    pn = np.zeros(g.N)

    def Ab(kind, p):
        lin = assemble(pb, p, pn, 0.01)
        return basis_operator(pb, kind, lin.rho, lin.c, pn, 0.01)

    # (B4) is pressure independent: built once, never again (Sec. 3)
    st = BasisState(wb)
    assert st.update(Ab(4, pn), 0.1) == ne
    assert st.update(Ab(4, rng.uniform(0, 1, g.N)), 0.1) == 0
    # theta < 0: no adaptivity, everything is rebuilt
    assert st.update(Ab(4, pn), -1.0) == ne
    # (B1): a huge threshold keeps the first build
    st1 = BasisState(wb)
    st1.update(Ab(1, pn), 1e30)
    assert st1.update(Ab(1, rng.uniform(0, 1, g.N)), 1e30) == 0
    # a change confined to one edge segment rebuilds it and everything above
    # it that depends on it, and nothing else
    st2 = BasisState(wb)
    A0 = Ab(4, pn)
    st2.update(A0, 0.1)
    edge = next(i for i, e in enumerate(wb.entities) if e.level == 1 and len(e.cells) > 1)
    A1 = A0.copy().tolil()
    c0 = wb.entities[edge].cells[0]
    A1[c0, c0] = A1[c0, c0] * 1.5
    n = st2.update(A1.tocsr(), 0.1)
    deps = st2._deps
    faces = {i for i, e in enumerate(wb.entities) if e.level == 2 and edge in deps[i]}
    inter = {i for i, e in enumerate(wb.entities) if e.level == 3 and deps[i] & faces}
    assert n == 1 + len(faces) + len(inter)
    # the adaptive result equals a full rebuild with the same operator
    full = prolongation(A1.tocsr(), wb).to_csr(wb.Nc)
    np.testing.assert_allclose(st2.matrix().toarray(), full.toarray(), atol=1e-14)


def test_newton_control_counts(rng):
    """Every linearisation runs at least one C-AMS iteration; the stopping
    test is on ||eps||_2 relative to the start of the step (Reading R13)."""
    g = _grid(10, 10, 1)
    pb = _problem(g, _lognormal(g.N, rng), c=0.5)
    opt = Options(coarse=(5, 5, 1), basis=4, n_post=1, nl_tol=1e-8)
    p, st = run(pb, opt, np.zeros(g.N), 0.002, 2)
    for s in st:
        assert s.converged and s.newton_its == len(s.cams_per_newton)
        assert all(c >= 1 for c in s.cams_per_newton)
        assert s.eps_hist[-1] < 1e-8 * s.eps_hist[0] <= s.eps_hist[-2]


def _iteration_matrix(A, P, R, lu, LU, n_post):
    """G with e -> G e the error propagation of one C-AMS iteration, built
    column by column from the oracle's own iteration on f = 0 (exact solution
    0, so the iterate is the error)."""
    n = A.shape[0]
    f0 = np.zeros(n)
    return np.column_stack([cams_iteration(A, f0, np.eye(n)[:, j], P, R, lu, LU, 0, n_post)
                            for j in range(n)])


@pytest.mark.parametrize("n_post", [1, 2])
def test_inner_stopping_rule_on_an_eigenvector(rng, n_post):
    """Sec. 4.1.1: the inner loop runs C-AMS iterations until
    ||r^i||_2 / ||r^0||_2 < 0.1, r^0 being the residual of the new
    linearisation before its first iteration.  On a linear problem (rho
    constant, one linearisation is exact) started at p* + v, v an eigenvector
    of the iteration matrix G for its largest eigenvalue lam (real, since
    MSFE and the symmetric ILU(0) factor make G similar to an A-self-adjoint
    operator), every iteration scales the error and the residual by lam, so
    the count is the smallest i with lam^i < 0.1.  Taking r^0 after the first
    iteration would give one more; comparing with the previous iterate, or
    a missed cap, would never stop before max_cams."""
    g = _grid(12, 10, 1)
    pb = _problem(g, _lognormal(g.N, rng), c=0.0)           # rho = 1: linear
    opt = Options(coarse=(3, 5, 1), basis=4, n_post=n_post, nl_tol=1e-30, max_newton=1,
                  max_cams=500)
    lin = assemble(pb, np.zeros(g.N), np.zeros(g.N), 0.01)
    A = lin.A.tocsr()
    assert abs(A - A.T).max() == 0.0
    wb = build_wirebasket(g, opt.coarse)
    P = prolongation(basis_operator(pb, 4, lin.rho, lin.c, np.zeros(g.N), 0.01), wb).to_csr(wb.Nc)
    R = restriction(0, P, wb)
    lu = coarse_factor(coarse_operator(R, A, P))
    LU = ilu0(A)
    G = _iteration_matrix(A, P, R, lu, LU, n_post)
    lam, V = np.linalg.eig(G)
    k = int(np.argmax(lam.real))
    lmax = lam[k].real
    assert abs(lam[k].imag) < 1e-12 and 0.2 < lmax < 0.99
    v = V[:, k].real
    v /= np.abs(v).max()
    count = int(np.ceil(np.log(0.1) / np.log(lmax)))
    assert lmax ** count < 0.1 * (1 - 1e-6) and lmax ** (count - 1) > 0.1 * (1 + 1e-6)
    pstar = spl.spsolve(A.tocsc(), lin.f)
    # the residual history of the oracle's loop follows lam^i
    p, hist = pstar + 1e-3 * v, []
    for _ in range(count + 1):
        hist.append(np.linalg.norm(lin.f - A @ p))
        p = cams_iteration(A, lin.f, p, P, R, lu, LU, 0, n_post)
    ratios = np.array(hist[1:]) / np.array(hist[:-1])
    np.testing.assert_allclose(ratios, lmax, rtol=1e-6)
    # the solver's inner loop stops at exactly that count
    state = BasisState(wb)
    _, st = solve_step(pb, wb, state, opt, np.zeros(g.N), 0.01, p_init=pstar + 1e-3 * v)
    assert st.cams_per_newton == [count]
    # and at the cap when the target is out of reach (and still re-linearises, R14)
    opt2 = Options(coarse=(3, 5, 1), basis=4, n_post=n_post, lin_rtol=1e-30, nl_tol=1e-30,
                   max_newton=2, max_cams=7)
    _, st2 = solve_step(pb, wb, BasisState(wb), opt2, np.zeros(g.N), 0.01, p_init=pstar + 1e-3 * v)
    assert st2.cams_per_newton == [7, 7] and not st2.converged


def test_msfe_then_msfv_closing_correction(rng):
    """Restriction 2 (Sec. 4.3): the step converges with MSFE exactly as with
    restriction 0, then one MSFV coarse correction of the last linearisation
    makes the restricted residual vanish block by block, without undoing the
    nonlinear convergence."""
    g = _grid(12, 10, 6)
    pb = _problem(g, _lognormal(g.N, rng, 2.0), c=0.2)
    wb0 = build_wirebasket(g, (4, 5, 3))
    p_n = np.zeros(g.N)
    dt = 0.01
    out = {}
    for R in (0, 2):
        opt = Options(coarse=(4, 5, 3), basis=4, restriction=R, n_post=2, nl_tol=1e-9)
        p, st = solve_step(pb, wb0, BasisState(wb0), opt, p_n, dt)
        out[R] = (p, st)
    (p0, s0), (p2, s2) = out[0], out[2]
    assert s0.converged and s2.converged and s2.msfv_final and not s0.msfv_final
    assert s2.newton_its == s0.newton_its and s2.cams_per_newton == s0.cams_per_newton
    # the correction is the MSFV coarse step on the linearisation at p0
    lin = assemble(pb, p0, p_n, dt)
    st = BasisState(wb0)
    st.update(basis_operator(pb, 4, lin.rho, lin.c, p_n, dt), 0.1)
    Rv = restriction(1, st.matrix(), wb0)
    blk = Rv @ (lin.f - lin.A @ p2)
    scale = np.abs(Rv @ np.abs(lin.A @ p0)).max()
    assert np.abs(blk).max() <= 1e-12 * scale
    # whereas the MSFE solution itself is not conservative on the blocks
    assert np.abs(Rv @ (lin.f - lin.A @ p0)).max() > 1e3 * np.abs(blk).max()
    e0 = np.linalg.norm(epsilon(pb, p0, p_n, dt))
    e2 = np.linalg.norm(epsilon(pb, p2, p_n, dt))
    assert e2 < 10 * e0 + 1e-12


# ------------------------------------ Test Case 2: prescribed cells, alpha --

def _tc2_problem(g, k, cells, vals, law=1, c=1.0, dirichlet=False):
    fl = Fluid(law, c, 1.0, 1.0, 0.1)
    bc = BC(dirichlet, 1.0, 0.0, fix_cell=np.asarray(cells), fix_value=np.asarray(vals))
    return Problem.build(g, fl, bc, *k)


def _columns(g, a, b):
    z = np.arange(g.nz)
    ca = a[0] + g.nx * (a[1] + g.ny * z)
    cb = b[0] + g.nx * (b[1] + g.ny * z)
    return np.concatenate([ca, cb]), np.concatenate([np.ones(g.nz), np.zeros(g.nz)])


@pytest.mark.parametrize("alpha", [1.0, 5.0])
def test_prescribed_columns_solve_the_mass_balance(rng, alpha):
    """Sec. 4.2.2 (Reading R19): with p prescribed on two vertical columns of
    cells, the converged step holds exactly those values there and is a root
    of the discrete mass balance (Eq. 2, evaluated by the flux-sum residual,
    not by the linear system) on every other cell."""
    nx, ny, nz = 12, 10, 8
    h = 1.0 / nx
    g = Grid(nx, ny, nz, alpha * h, h, h)
    cells, vals = _columns(g, (0, 0), (nx - 1, ny - 1))
    pb = _tc2_problem(g, _lognormal(g.N, rng, 2.0), cells, vals)
    p_n = np.zeros(g.N)
    dt = 0.4 * 0.1 * alpha ** 2
    opt = Options(coarse=(4, 5, 4), basis=4, n_post=5, nl_tol=1e-12, max_newton=30)
    p, st = run(pb, opt, p_n, dt, 1)
    assert st[0].converged
    assert np.array_equal(p[cells], vals)
    free = np.ones(g.N, bool)
    free[cells] = False
    F0 = residual(pb, pb.with_fixed(p_n), p_n, dt)
    F = residual(pb, p, p_n, dt)
    assert np.abs(F[free]).max() < 1e-9 * np.abs(F0[free]).max()
    # the columns drive flow from the p = 1 column to the p = 0 column
    assert 0.0 < p[free].min() and p[free].max() < 1.0
    assert p[0 + nx * 1] > p[(nx - 1) + nx * (ny - 2)]


def test_prescribing_the_solution_changes_nothing(rng):
    """Fixing interior cells at the values the unconstrained problem takes
    there leaves the solution unchanged: the elimination adds nothing but
    the known values (a wrong sign or a lost coupling would move it)."""
    g = _grid(12, 10, 6)
    k = _lognormal(g.N, rng, 1.5)
    p_n = np.zeros(g.N)
    dt = 0.01
    opt = Options(coarse=(4, 5, 3), basis=4, n_post=3, nl_tol=1e-12, max_newton=30)
    pb0 = _problem(g, k, law=0, c=0.3)
    p_ref, st = run(pb0, opt, p_n, dt, 1)
    assert st[0].converged
    z = np.arange(g.nz)
    cells = np.concatenate([3 + g.nx * (4 + g.ny * z), 9 + g.nx * (8 + g.ny * z)])
    fl = Fluid(0, 0.3, 1.0, 1.0, 0.1)
    bc = BC(True, 1.0, 0.0, fix_cell=cells, fix_value=p_ref[cells])
    pb1 = Problem.build(g, fl, bc, *k)
    p_fix, st1 = run(pb1, opt, p_n, dt, 1)
    assert st1[0].converged
    np.testing.assert_allclose(p_fix, p_ref, rtol=0, atol=1e-9)
    # whereas fixing them elsewhere does move it
    bc2 = BC(True, 1.0, 0.0, fix_cell=cells, fix_value=p_ref[cells] + 0.1)
    p_off, _ = run(Problem.build(g, fl, bc2, *k), opt, p_n, dt, 1)
    assert np.abs(p_off - p_ref).max() > 1e-3


def test_prescribed_cells_leave_a_symmetric_system_and_zero_basis_rows(rng):
    """Reading R19: the eliminated A and A_b stay symmetric, fixed rows are
    unit rows, and the basis functions vanish on fixed cells; the coarse
    operator P^T A P stays symmetric positive definite."""
    g = _grid(12, 10, 8)
    cells, vals = _columns(g, (0, 0), (11, 9))
    pb = _tc2_problem(g, _lognormal(g.N, rng, 2.0), cells, vals)
    p_n = np.zeros(g.N)
    lin = assemble(pb, p_n, p_n, 0.04)
    A = lin.A.toarray()
    np.testing.assert_array_equal(A, A.T)
    np.testing.assert_array_equal(A[cells], np.eye(g.N)[cells])
    np.testing.assert_array_equal(lin.f[cells], vals)
    assert np.all(lin.eps[cells] == 0.0)
    wb = build_wirebasket(g, (4, 5, 4))
    Ab = basis_operator(pb, 4, lin.rho, lin.c, p_n, 0.04)
    Abd = Ab.toarray()
    np.testing.assert_array_equal(Abd, Abd.T)
    P = prolongation(Ab, wb).to_csr(wb.Nc).toarray()
    assert np.all(P[cells] == 0.0)
    Ac = P.T @ A @ P
    np.testing.assert_allclose(Ac, Ac.T, rtol=1e-12, atol=1e-14 * np.abs(Ac).max())
    assert np.linalg.eigvalsh(0.5 * (Ac + Ac.T)).min() > 0
    # the basis still sums to one away from the columns' dual blocks
    far = (np.abs(g.coords()[0] - 6) <= 1) & (np.abs(g.coords()[1] - 5) <= 1)
    np.testing.assert_allclose(P.sum(axis=1)[far], 1.0, rtol=1e-12)


def test_prescribed_coarse_node_is_rejected():
    """A fixed cell may not be a coarse node (Reading R19)."""
    g = _grid(8, 8, 1)
    wb = build_wirebasket(g, (4, 4, 1))
    node = int(np.flatnonzero(wb.level == 0)[0])
    one = np.ones(g.N)
    pb = _tc2_problem(g, (one, one, one), [node], [0.5])
    with pytest.raises(ValueError):
        run(pb, Options(coarse=(4, 4, 1)), np.zeros(g.N), 0.01, 1)


@pytest.mark.parametrize("alpha", [5.0, 10.0])
def test_stretched_grid_closed_forms(alpha):
    """Delta x / alpha = Delta y = Delta z: for homogeneous k the face
    transmissibilities are k dy dz / dx and k dx dz / dy, so T_x / T_y =
    1 / alpha^2; and the incompressible west-east solution is still
    p_i = 1 - (x_i + 1/2)/nx, which C-AMS reaches."""
    nx, ny, nz = 12, 8, 6
    h = 1.0 / nx
    g = Grid(nx, ny, nz, alpha * h, h, h)
    one = np.ones(g.N)
    pb = _problem(g, (one, one, one), law=1, c=0.0)
    fc = pb.faces
    d = fc.hi - fc.lo
    tx, ty, tz = fc.T[d == 1], fc.T[d == nx], fc.T[d == nx * ny]
    np.testing.assert_allclose(tx, h * h / (alpha * h), rtol=1e-14)
    np.testing.assert_allclose(ty, alpha * h * h / h, rtol=1e-14)
    np.testing.assert_allclose(tx[0] / ty[0], 1.0 / alpha ** 2, rtol=1e-14)
    np.testing.assert_allclose(tz, ty[0], rtol=1e-14)
    opt = Options(coarse=(2, 4, 3), basis=4, n_post=3, nl_tol=1e-13, max_newton=20)
    p, st = run(pb, opt, np.zeros(g.N), 1e-3, 1)
    x, _, _ = g.coords()
    np.testing.assert_allclose(p, 1.0 - (x + 0.5) / g.nx, atol=1e-12)
    assert st[0].converged


# ------------------------------------------- the learned surrogate's network --

def test_net_conv_matches_brute_force(rng):
    """The oracle's convolution against the defining sum written as loops,
    with zero padding; a single centre tap of weight 1 is the identity and an
    off-centre tap a shift."""
    from oracle.net import conv_forward
    B, ci, co, S = 2, 3, 2, 4
    x = rng.standard_normal((B, ci, S, S, S))
    w = rng.standard_normal((co, ci, 27))
    b = rng.standard_normal(co)
    y = conv_forward(x, w, b, relu=False)
    ref = np.zeros_like(y)
    for bb in range(B):
        for o in range(co):
            for z in range(S):
                for yy in range(S):
                    for xx in range(S):
                        s = b[o]
                        for i in range(ci):
                            for t in range(27):
                                dx, dy, dz = t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1
                                u, v, q = xx + dx, yy + dy, z + dz
                                if 0 <= u < S and 0 <= v < S and 0 <= q < S:
                                    s += w[o, i, t] * x[bb, i, q, v, u]
                        ref[bb, o, z, yy, xx] = s
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)
    wi = np.zeros((1, 1, 27)); wi[0, 0, 13] = 1.0
    np.testing.assert_array_equal(conv_forward(x[:, :1], wi, np.zeros(1), False), x[:, :1])
    ws = np.zeros((1, 1, 27)); ws[0, 0, 14] = 1.0                    # dx = +1
    sh = conv_forward(x[:, :1], ws, np.zeros(1), False)
    np.testing.assert_array_equal(sh[..., :-1], x[:, :1, :, :, 1:])
    assert np.all(sh[..., -1] == 0.0)


def test_net_gradients_match_finite_differences(rng):
    """Backward pass of a 3-layer network (ReLU between layers) against
    central finite differences of the masked MSE loss."""
    from oracle.net import mse, network_backward, network_forward
    S, B = 4, 2
    chans = [2, 3, 3, 2]
    layers = [(0.4 * rng.standard_normal((chans[k + 1], chans[k], 27)),
               0.1 * rng.standard_normal(chans[k + 1])) for k in range(3)]
    x = rng.standard_normal((B, chans[0], S, S, S))
    target = rng.standard_normal((B, chans[-1], S, S, S))
    mask = (rng.random((B, chans[-1], S, S, S)) < 0.6).astype(float)
    count = mask.sum()

    def loss(ls):
        y, _ = network_forward(x, ls)
        return mse(y, target, mask, count)[0]

    y, acts = network_forward(x, layers)
    _, gy = mse(y, target, mask, count)
    grads = network_backward(acts, layers, gy)
    h = 1e-6
    for k in range(3):
        for which in (0, 1):
            arr = layers[k][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h; lp = loss(layers)
                flat[idx] = old - h; lm = loss(layers)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[k][which].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, which, idx, fd, an)


def test_net_adam_first_step_is_signed_lr():
    """With zero moments the first Adam step moves each parameter by
    -lr * g / (|g| + eps): the sign step of size lr (bias correction)."""
    from oracle.net import adam_step
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p, m, v = adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 0.01, 0.9, 0.999, 1e-12, 1)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-9, atol=1e-12)


def test_net_energy_loss_gradient_and_null_space(rng):
    """The energy loss's gradient against finite differences, and two facts
    of the norm: a constant error on a patch whose boundary error is zero is
    not free (the boundary pins it), and with unit couplings the energy of a
    single unit error is the number of its interior-facing plus boundary
    faces (six for an inner cell)."""
    from oracle.net import energy_loss
    B, C, S = 2, 3, 5
    x = rng.standard_normal((B, 3, S, S, S))
    t = rng.standard_normal((B, C, S, S, S))
    mask = np.zeros((B, C, S, S, S)); mask[:, :, 1:-1, 1:-1, 1:-1] = 1.0
    p = t + 0.1 * rng.standard_normal(t.shape)
    E, g = energy_loss(p, t, mask, x)
    h = 1e-6
    for idx in [(0, 1, 2, 2, 2), (1, 0, 1, 3, 2), (0, 2, 3, 1, 1), (1, 1, 0, 2, 2)]:
        pp = p.copy(); pp[idx] += h
        pm = p.copy(); pm[idx] -= h
        fd = (energy_loss(pp, t, mask, x)[0] - energy_loss(pm, t, mask, x)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd))
    assert g[1, 1, 0, 2, 2] == 0.0                       # boundary entries carry no gradient
    e1 = np.zeros_like(t); e1[0, 0, 2, 2, 2] = 1.0
    E1, _ = energy_loss(t + e1, t, mask, np.zeros_like(x))
    np.testing.assert_allclose(E1 * mask.sum(), 6.0)
    const = np.where(mask > 0, 1.0, 0.0)
    assert energy_loss(t + const, t, mask, np.zeros_like(x))[0] > 0.0


# -------------------------------------------- correction functions (A14) --

def _reduced_system(Ab, wb):
    """The whole block-triangular reduced system in the natural order (same
    construction as the global prolongation): an independent route."""
    N = wb.grid.N
    coo = Ab.tocoo()
    r, c, v = coo.row, coo.col, coo.data
    lr, lc = wb.level[r], wb.level[c]
    keep = (r != c) & ((lc == lr) | (lc == lr - 1)) & (lr > 0)
    lump = (r != c) & (lc == lr + 1) & (lr > 0)
    diag = np.where(wb.level > 0, Ab.diagonal(), 1.0) + np.bincount(r[lump], weights=v[lump], minlength=N)
    return sp.csc_matrix((np.concatenate([v[keep], diag]),
                          (np.concatenate([r[keep], np.arange(N)]), np.concatenate([c[keep], np.arange(N)]))),
                         shape=(N, N))


@pytest.mark.parametrize("shape,coarse", [((12, 10, 1), (4, 5, 1)), ((12, 10, 6), (4, 5, 3))])
def test_correction_function_equals_the_global_reduced_solve(rng, shape, coarse):
    """Reading R21: the staged local solves with the residual as source equal
    one solve of the global reduced system whose vertex rows are zero."""
    from oracle.basis import correction_function
    g = _grid(*shape)
    pb = _problem(g, _lognormal(g.N, rng, 1.5))
    lin = assemble(pb, np.zeros(g.N), np.zeros(g.N), 0.01)
    wb = build_wirebasket(g, coarse)
    Ab = basis_operator(pb, 1, lin.rho, lin.c, np.zeros(g.N), 0.01)
    r = rng.standard_normal(g.N)
    psi = correction_function(Ab, wb, r)
    rhs = r.copy(); rhs[wb.vertex_cell] = 0.0
    ref = spl.spsolve(_reduced_system(Ab, wb), rhs)
    np.testing.assert_allclose(psi, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert np.all(psi[wb.vertex_cell] == 0.0)


def test_correction_function_with_msfe_is_exact_in_1d(rng):
    """1D, no-flow ends, compressible with the (B1) basis operator, which is
    then A itself: the local problems between vertices decouple, the basis
    functions are A-orthogonal to every function that vanishes on the
    vertices, so one correction-function stage followed by the MSFE stage (no
    smoothing) returns the exact solution of A p = f from any start."""
    from oracle.basis import correction_function
    n = 24
    g = Grid(n, 1, 1, 1.0 / n, 1.0, 1.0)
    k = np.exp(1.5 * rng.standard_normal(n))
    pb = _problem(g, (k, k, k), law=0, c=0.2, dirichlet=False)
    p_nu = rng.uniform(0, 1, n)
    lin = assemble(pb, p_nu, np.zeros(n), 0.01)
    wb = build_wirebasket(g, (6, 1, 1))
    Ab = basis_operator(pb, 1, lin.rho, lin.c, np.zeros(n), 0.01)
    np.testing.assert_allclose(Ab.toarray(), lin.A.toarray(), rtol=1e-13, atol=1e-15)
    P = prolongation(Ab, wb).to_csr(wb.Nc)
    R = restriction(0, P, wb)
    lu = coarse_factor(coarse_operator(R, lin.A, P))
    p0 = rng.standard_normal(n)
    p1 = cams_iteration(lin.A, lin.f, p0, P, R, lu, ilu0(lin.A), 0, 0,
                        cf=lambda r: correction_function(Ab, wb, r))
    exact = spl.spsolve(lin.A.tocsc(), lin.f)
    np.testing.assert_allclose(p1, exact, rtol=1e-10, atol=1e-12 * np.abs(exact).max())
    # without the correction function one iteration is not exact
    p2 = cams_iteration(lin.A, lin.f, p0, P, R, lu, ilu0(lin.A), 0, 0)
    assert np.abs(p2 - exact).max() > 1e-3 * np.abs(exact).max()


def test_correction_function_is_local_and_keeps_the_fixed_point(rng):
    """A residual inside one dual-block interior gives a correction function
    supported on that interior only; with correction functions on, the step
    converges to the same pressure as without."""
    from oracle.basis import correction_function
    g = _grid(12, 10, 1)
    pb = _problem(g, _lognormal(g.N, rng, 1.5), c=0.2)
    wb = build_wirebasket(g, (4, 5, 1))
    lin = assemble(pb, np.zeros(g.N), np.zeros(g.N), 0.01)
    Ab = basis_operator(pb, 4, lin.rho, lin.c, np.zeros(g.N), 0.01)
    interior = [e for e in wb.entities if e.level == wb.d_active and len(e.cells) > 1][0]
    r = np.zeros(g.N); r[interior.cells[0]] = 1.0
    psi = correction_function(Ab, wb, r)
    assert set(np.flatnonzero(psi)) <= set(interior.cells.tolist())
    assert psi[interior.cells[0]] != 0.0
    out = []
    for cf in (False, True):
        opt = Options(coarse=(4, 5, 1), basis=4, n_post=1, nl_tol=1e-11, cf=cf, max_newton=30)
        p, st = run(pb, opt, np.zeros(g.N), 0.01, 1)
        assert st[0].converged
        out.append(p)
    np.testing.assert_allclose(out[1], out[0], rtol=0, atol=1e-8)


# ---------------------------------------------- full-Jacobian Newton (R22) --

@pytest.mark.parametrize("law,c", [(0, 0.8), (1, 0.5)])
def test_full_jacobian_matches_finite_differences(rng, law, c):
    """Reading R22: the full-Jacobian matrix is V rho_i^nu times the
    derivative of the paper's equation in volume units (the mass residual
    over V rho), here taken by central differences of the residual function
    (heterogeneous, Dirichlet faces, wells, uneven pressure).  The lagged
    matrix of Eq. 3 misses it by far more than the difference error.  At rest
    (no-flow, uniform pressure) and for an incompressible fluid both agree."""
    g = _grid(5, 4, 3)
    k = _lognormal(g.N, rng, 1.0)
    src = (np.array([3, g.N - 2]), np.array([0.3, -0.2]))
    pb = _problem(g, k, law=law, c=c, src=src)
    p = rng.uniform(0.0, 1.0, g.N)
    pn = rng.uniform(0.0, 1.0, g.N)
    dt = 0.05
    G = lambda q: residual(pb, q, pn, dt) / (g.V * pb.fluid.rho(q))
    h = 1e-6
    J = np.zeros((g.N, g.N))
    for j in range(g.N):
        e = np.zeros(g.N); e[j] = h
        J[:, j] = (G(p + e) - G(p - e)) / (2 * h)
    J *= (g.V * pb.fluid.rho(p))[:, None]
    full = assemble(pb, p, pn, dt, full_jacobian=True).A.toarray()
    lag = assemble(pb, p, pn, dt).A.toarray()
    scale = np.abs(J).max()
    np.testing.assert_allclose(full, J, rtol=0, atol=1e-7 * scale)
    assert np.abs(lag - J).max() > 1e-3 * scale
    # at rest the flux and its density derivative vanish
    pbr = _problem(g, k, law=law, c=c, dirichlet=False)
    u = np.full(g.N, 0.7)
    np.testing.assert_array_equal(assemble(pbr, u, pn, dt, True).A.toarray(),
                                  assemble(pbr, u, pn, dt).A.toarray())
    pbi = _problem(g, k, law=1, c=0.0, src=src)
    np.testing.assert_array_equal(assemble(pbi, p, pn, dt, True).A.toarray(),
                                  assemble(pbi, p, pn, dt).A.toarray())


def _newton_norms(pb, pn, dt, full):
    """||F|| / ||F_0|| along Newton steps with exact linear solves."""
    p = pn.copy()
    hist = []
    for _ in range(40):
        hist.append(float(np.linalg.norm(residual(pb, p, pn, dt))))
        if hist[-1] < 1e-13 * hist[0]:
            break
        lin = assemble(pb, p, pn, dt, full)
        p = spl.spsolve(lin.A.tocsc(), lin.f)
    return np.array(hist) / hist[0], p


@pytest.mark.parametrize("law,c", [(0, 2.0), (1, 0.8)])
def test_full_jacobian_newton_is_quadratic(rng, law, c):
    """Reading R22: with exact linear solves the full-Jacobian step converges
    at order 2 (the last error-reduction exponents log(e_{k+1}/e_k) /
    log(e_k/e_{k-1}) near 2), while the lagged step of Eq. 3 converges at
    order 1; both reach the same root."""
    g = _grid(8, 6, 1)
    k = _lognormal(g.N, rng, 1.0)
    pb = _problem(g, k, law=law, c=c)
    pn = np.zeros(g.N)
    order = lambda e: np.log(e[2:] / e[1:-1]) / np.log(e[1:-1] / e[:-2])
    ef, pf = _newton_norms(pb, pn, 1.0, True)
    el, pl = _newton_norms(pb, pn, 1.0, False)
    tail = ef[ef > 1e-12]
    assert 1.8 < order(tail)[-1] < 2.3
    assert np.median(order(el[el > 1e-12])[-4:]) < 1.2
    assert ef.size < el.size
    np.testing.assert_allclose(pf, pl, rtol=0, atol=1e-12)


@pytest.mark.parametrize("restriction", [0, 1])
def test_full_jacobian_cams_step_reaches_the_same_root(rng, restriction):
    """The C-AMS solve of a full-Jacobian (nonsymmetric) linearisation, with
    a fixed cell and a well, converges to the pressure the lagged step finds,
    in no more Newton steps."""
    g = _grid(12, 10, 1)
    k = _lognormal(g.N, rng, 1.5)
    bc = BC(True, 1.0, 0.0, np.array([25]), np.array([0.05]), np.array([62]), np.array([0.4]))
    pb = Problem.build(g, Fluid(0, 1.5, 1.0, 1.0, 0.1), bc, *k)
    out = []
    for full in (False, True):
        opt = Options(coarse=(4, 5, 1), basis=1, restriction=restriction, n_post=2,
                      nl_tol=1e-11, full_jacobian=full, max_newton=60)
        p, st = run(pb, opt, np.zeros(g.N), 0.2, 1)
        assert st[0].converged
        out.append((p, st[0].newton_its))
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=0, atol=1e-9)
    assert out[1][1] <= out[0][1]
    assert out[1][0][62] == 0.4


def test_correction_functions_destabilise_large_3d_blocks(rng):
    """Sec. 4.1.4 finds the iteration with correction functions unstable.
    A mechanism: for an error e that is smooth along a face patch of b x b
    cells (unit couplings w), A e ~ (2 pi^2 w / b^2 + 2 w) e, the in-face
    Laplacian plus the two transverse couplings, while the face's lumped
    operator keeps the in-face part only; Psi then overshoots e by about
    b^2 / pi^2.  With blocks of 10^3 cells (~10) the iteration with one
    ILU(0) step diverges even on a homogeneous field and converges without
    correction functions; with 2^3 blocks both converge."""
    from oracle.basis import correction_function
    out = {}
    for n, b in ((20, 10), (8, 2)):
        g = _grid(n, n, n)
        one = np.ones(g.N)
        pb = _problem(g, (one, one, one), c=0.1)
        p_nu = rng.uniform(0, 1, g.N)
        lin = assemble(pb, p_nu, np.zeros(g.N), 0.01)
        wb = build_wirebasket(g, (b, b, b))
        Ab = basis_operator(pb, 4, lin.rho, lin.c, np.zeros(g.N), 0.01)
        P = prolongation(Ab, wb).to_csr(wb.Nc)
        R = restriction(0, P, wb)
        lu = coarse_factor(coarse_operator(R, lin.A, P))
        LU = ilu0(lin.A)
        for cf in (False, True):
            p = np.zeros(g.N)
            r0 = np.linalg.norm(lin.f)
            for _ in range(6):
                p = cams_iteration(lin.A, lin.f, p, P, R, lu, LU, 0, 1,
                                   (lambda r: correction_function(Ab, wb, r)) if cf else None)
            out[(b, cf)] = np.linalg.norm(lin.f - lin.A @ p) / r0
    assert out[(10, False)] < 0.1 and out[(10, True)] > 10.0
    assert out[(2, False)] < 0.1 and out[(2, True)] < 0.1
