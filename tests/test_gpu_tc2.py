"""Test Case 2 of Sec. 4.2.2 on the GPU against the oracle: pressure
prescribed at the centres of two vertical columns of cells (eliminated
symmetrically, Reading R19), stretched grids Delta x / alpha = Delta y =
Delta z with alpha in {1, 5, 10}, coarsening 8x8x8 (alpha 1) and 2x8x8.

Tolerances as in the other parity tests: single-pass arithmetic at
1e-13..1e-11 relative, P within the local-condition bound, pressures after
a few C-AMS iterations at 1e-10, converged pressures at 1e-9 (FP64) and
1e-6 (mixed precision), Newton counts within one.  The prescribed values
are held exactly: a fixed row is a unit row with a zero residual, so no
stage ever moves p there."""
import numpy as np
import pytest

import oracle
from oracle.basis import basis_operator, prolongation
from oracle.coarse import coarse_factor, coarse_operator, restriction
from oracle.ilu import ilu0
from oracle.solver import cams_iteration
from oracle.wirebasket import build_wirebasket

from _cases import coarse_from_gpu, gpu_handle, make_case, matrix_from_gpu, p_from_gpu
from test_gpu_parity import _rel, p_tolerance

pytestmark = pytest.mark.gpu

SMALL = {
    1: dict(nx=24, ny=24, nz=16),     # coarse 8x8x8 -> 3x3x2 coarse nodes
    5: dict(nx=16, ny=16, nz=16),     # coarse 2x8x8 -> 8x2x2
    10: dict(nx=20, ny=24, nz=16),    # coarse 2x8x8 -> 10x3x2
}


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _case(alpha, **kw):
    return make_case(f"3d-64x64x64-lines-a{alpha}", **{**SMALL[alpha], **kw})


@pytest.mark.parametrize("alpha", [1, 5, 10])
def test_tc2_operators_and_iterations(cams, alpha):
    """Assembly with the eliminated columns, P, R A P, the ILU(0) pivots
    and four C-AMS iterations, element by element."""
    case = _case(alpha)
    N = case.N
    h, bc, keep = gpu_handle(case)
    try:
        rng = np.random.default_rng(11)
        p_nu, p_n = rng.uniform(-0.1, 1.1, N), rng.uniform(-0.1, 1.1, N)
        dt = case.inp["dt"]
        cams.cams_assemble(h, p_nu, p_n, dt, bc)
        lin = oracle.assemble(case.pb, p_nu, p_n, dt)
        Ad, Ax, Ay, Az = matrix_from_gpu(h, N)
        assert _rel(Ad, lin.A.diagonal()) < 1e-13
        i = np.arange(N)
        nx, ny = case.w.nx, case.w.ny
        for arr, off, ok in ((Ax, 1, i % nx > 0), (Ay, nx, (i // nx) % ny > 0),
                             (Az, nx * ny, i // (nx * ny) > 0)):
            ref = np.zeros(N)
            ref[ok] = np.asarray(lin.A[i[ok], i[ok] - off]).ravel()
            assert _rel(arr, ref) < 1e-13
        assert _rel(cams.cams_get(h, cams.CAMS_Q_RHS, np.zeros(N)), lin.f) < 1e-12
        eps = cams.cams_get(h, cams.CAMS_Q_EPS, np.zeros(N))
        assert _rel(eps, lin.eps) < 1e-11
        fc = case.inp["fix_cell"]
        assert np.all(eps[fc] == 0.0)
        pg0 = cams.cams_get(h, cams.CAMS_Q_PRESSURE, np.zeros(N))
        assert np.array_equal(pg0[fc], case.inp["fix_value"])

        cams.cams_update_basis(h, True)
        wb = build_wirebasket(case.pb.grid, case.w.coarse)
        p_ref = case.pb.with_fixed(p_nu)
        Ab = basis_operator(case.pb, case.w.basis, lin.rho, lin.c, p_n, dt)
        P = prolongation(Ab, wb).to_csr(wb.Nc)
        Pg, _, _ = p_from_gpu(h, N, wb.Nc)
        tol = p_tolerance(Ab, wb)
        assert np.abs((Pg - P).toarray()).max() < tol
        assert np.all(Pg.toarray()[fc] == 0.0)
        Ac, _ = coarse_from_gpu(h, wb.nc)
        Rm = restriction(0, P, wb)
        Aco = np.asarray(coarse_operator(Rm, lin.A, P))
        assert _rel(Ac, Aco) < 1e-13 + 4 * tol
        assert np.array_equal(Ac, Ac.T)
        d = cams.cams_get(h, cams.CAMS_Q_ILU_DIAG, np.zeros(N))
        LU = ilu0(lin.A)
        assert _rel(d, LU[1].diagonal()) < 1e-12

        res = cams.cams_iterate(h, 4)
        pg = cams.cams_get(h, cams.CAMS_Q_PRESSURE, np.zeros(N))
        lu = coarse_factor(coarse_operator(Rm, lin.A, P))
        p = p_ref.copy()
        ro = [np.linalg.norm(lin.f - lin.A @ p)]
        for _ in range(4):
            p = cams_iteration(lin.A, lin.f, p, P, Rm, lu, LU, 0, case.w.n_post)
            ro.append(np.linalg.norm(lin.f - lin.A @ p))
        assert _rel(pg, p) < 1e-10
        assert np.array_equal(pg[fc], case.inp["fix_value"])
        np.testing.assert_allclose(res, ro, rtol=1e-7)
    finally:
        cams.cams_destroy(h)


_ORACLE = {}


def _oracle_step(case):
    """The oracle's step, shared by the FP64 and mixed-precision tests (the
    oracle does not depend on the engine's precision)."""
    w = case.w
    key = (w.name, w.nx, w.ny, w.nz, w.nl_tol)
    if key not in _ORACLE:
        q, sto = oracle.run(case.pb, case.opt, case.inp["p0"], case.inp["dt"], 1)
        _ORACLE[key] = (q, sto)
    return _ORACLE[key]


def _solve(cams, case):
    h, bc, keep = gpu_handle(case)
    try:
        p = case.inp["p0"].copy()
        st = cams.cams_solve(h, case.inp["p0"].copy(), case.inp["dt"], bc, p)
    finally:
        cams.cams_destroy(h)
    return p, st


@pytest.mark.parametrize("alpha", [1, 5, 10])
@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_tc2_step_matches_oracle(cams, alpha, precision, tol):
    """One implicit step t* = 0 -> 0.4 on the scaled-down grids."""
    case = _case(alpha, precision=precision, nl_tol=1e-8)
    p, st = _solve(cams, case)
    q, sto = _oracle_step(case)
    assert st.converged and sto[0].converged
    assert _rel(p, q) < tol
    assert abs(st.newton_its - sto[0].newton_its) <= 1
    if precision == 0:
        assert abs(st.cams_its - sto[0].cams_its) <= max(1, st.newton_its)
    else:
        assert st.cams_its <= 2 * sto[0].cams_its + 2 * st.newton_its
    assert np.array_equal(p[case.inp["fix_cell"]], case.inp["fix_value"])


@pytest.mark.parametrize("alpha", [1, 5, 10])
@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_tc2_full_size_matches_oracle(cams, alpha, precision, tol):
    """The full 64^3 workloads, in the configuration the benchmark times,
    against the oracle run on the same inputs (about 20 s each on the CPU)."""
    case = make_case(f"3d-64x64x64-lines-a{alpha}", precision=precision)
    p, st = _solve(cams, case)
    q, sto = _oracle_step(case)
    assert st.converged and sto[0].converged
    assert _rel(p, q) < tol
    assert abs(st.newton_its - sto[0].newton_its) <= 1
    assert np.array_equal(p[case.inp["fix_cell"]], case.inp["fix_value"])


def test_tc2_rejects_a_fixed_coarse_node(cams):
    """A prescribed cell on a coarse node is refused with CAMS_EINVAL."""
    case = _case(5)
    h, bc, keep = gpu_handle(case)
    try:
        # (1, 4, 4) is a coarse node of the 2x8x8 coarsening (offsets 1, 4, 4)
        node = 1 + case.w.nx * (4 + case.w.ny * 4)
        bc2, keep2 = cams.make_bc(False, 1.0, 0.0, None, None,
                                  np.array([node], np.int32), np.array([0.5]))
        p = case.inp["p0"].copy()
        with pytest.raises(cams.CamsError) as e:
            cams.cams_solve(h, p.copy(), case.inp["dt"], bc2, p)
        assert e.value.code == cams.CAMS_EINVAL
    finally:
        cams.cams_destroy(h)
