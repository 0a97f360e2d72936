"""The full-Jacobian Newton step (cams_options.jacobian = 1) on the GPU
against the oracle's Reading R22 (assemble(..., full_jacobian=True),
Options.full_jacobian): the nonsymmetric matrix entry by entry (lower and
transposed couplings), the nonsymmetric R A P (MSFE and MSFV), the ILU(0)
pivots, C-AMS iterates, and whole steps in FP64 and mixed precision.

Tolerances as in the symmetric parity tests: single-pass arithmetic at
1e-13..1e-11 relative, R A P within the local-condition bound of P, iterates
at 1e-10, converged pressures at 1e-9 (FP64) and 1e-6 (mixed precision)
with Newton counts within one."""
import numpy as np
import pytest

import oracle
from oracle.basis import basis_operator, prolongation
from oracle.coarse import coarse_factor, coarse_operator, restriction
from oracle.ilu import ilu0
from oracle.solver import cams_iteration
from oracle.wirebasket import build_wirebasket

from _cases import coarse_from_gpu, gpu_handle, make_case, matrix_from_gpu
from test_gpu_parity import _rel, p_tolerance

pytestmark = pytest.mark.gpu

CASES = {
    "2d-40x40": dict(name="2d-40x40"),
    "3d-wells-20x20x10": dict(name="3d-100x100x50-wells", nx=20, ny=20, nz=10, coarse=(5, 5, 5)),
    "3d-12x8x6-b2x4x3": dict(name="3d-200x200x100", nx=12, ny=8, nz=6, coarse=(2, 4, 3)),
    "tc2-a5-16": dict(name="3d-64x64x64-lines-a5", nx=16, ny=16, nz=16),
}


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _pressures(case, seed=7):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.2, 1.1, case.N), rng.uniform(-0.2, 1.1, case.N)


@pytest.mark.parametrize("cname", list(CASES))
def test_full_jacobian_assembly(cams, cname):
    case = make_case(**CASES[cname])
    h, bc, keep = gpu_handle(case, jacobian=1)
    try:
        N, nx, ny = case.N, case.w.nx, case.w.ny
        p_nu, p_n = _pressures(case)
        dt = case.inp["dt"]
        if len(case.inp["fix_cell"]):
            p_nu[case.inp["fix_cell"]] = case.inp["fix_value"]
        cams.cams_assemble(h, p_nu, p_n, dt, bc)
        lin = oracle.assemble(case.pb, p_nu, p_n, dt, full_jacobian=True)
        A = lin.A
        Ad, Ax, Ay, Az = matrix_from_gpu(h, N)
        up = cams.cams_get(h, cams.CAMS_Q_MATRIX_UPPER, np.zeros(3 * N))
        assert _rel(Ad, A.diagonal()) < 1e-13
        i = np.arange(N)
        for k, (arr, off, ok) in enumerate(((Ax, 1, i % nx > 0), (Ay, nx, (i // nx) % ny > 0),
                                            (Az, nx * ny, i // (nx * ny) > 0))):
            lo = np.zeros(N)
            lo[ok] = np.asarray(A[i[ok], i[ok] - off]).ravel()
            tr = np.zeros(N)
            tr[ok] = np.asarray(A[i[ok] - off, i[ok]]).ravel()
            assert _rel(arr, lo) < 1e-13
            assert _rel(up[k * N:(k + 1) * N], tr) < 1e-13
        assert abs(A - A.T).max() > 1e-6 * abs(A).max()       # the case is not symmetric
        f = cams.cams_get(h, cams.CAMS_Q_RHS, np.zeros(N))
        assert _rel(f, lin.f) < 1e-12
    finally:
        cams.cams_destroy(h)


@pytest.mark.parametrize("R", [0, 1])
@pytest.mark.parametrize("cname", ["2d-40x40", "3d-wells-20x20x10", "3d-12x8x6-b2x4x3"])
def test_full_jacobian_operators_and_iterations(cams, cname, R):
    case = make_case(**CASES[cname], restriction=R, n_pre=0, n_post=2)
    h, bc, keep = gpu_handle(case, jacobian=1)
    try:
        N = case.N
        p_nu, p_n = _pressures(case)
        dt = case.inp["dt"]
        cams.cams_assemble(h, p_nu, p_n, dt, bc)
        cams.cams_update_basis(h, True)
        wb = build_wirebasket(case.pb.grid, case.w.coarse)
        lin = oracle.assemble(case.pb, p_nu, p_n, dt, full_jacobian=True)
        Ab = basis_operator(case.pb, case.w.basis, lin.rho, lin.c, p_n, dt)
        P = prolongation(Ab, wb).to_csr(wb.Nc)
        Rm = restriction(R, P, wb)
        Ac = coarse_operator(Rm, lin.A, P)
        G, st = coarse_from_gpu(h, wb.nc)
        assert _rel(G, Ac) < 1e-13 + 4 * p_tolerance(Ab, wb)
        LU = ilu0(lin.A)
        d = cams.cams_get(h, cams.CAMS_Q_ILU_DIAG, np.zeros(N))
        assert _rel(d, LU[1].diagonal()) < 1e-12
        res = cams.cams_iterate(h, 3)
        pg = cams.cams_get(h, cams.CAMS_Q_PRESSURE, np.zeros(N))
        lu = coarse_factor(Ac)
        p = p_nu.copy()
        ro = [np.linalg.norm(lin.f - lin.A @ p)]
        for _ in range(3):
            p = cams_iteration(lin.A, lin.f, p, P, Rm, lu, LU, 0, 2)
            ro.append(np.linalg.norm(lin.f - lin.A @ p))
        assert _rel(pg, p) < 1e-10
        np.testing.assert_allclose(res, ro, rtol=1e-7)
    finally:
        cams.cams_destroy(h)


@pytest.mark.parametrize("cname,R", [("3d-12x8x6-b2x4x3", 0), ("3d-12x8x6-b2x4x3", 1),
                                     ("tc2-a5-16", 0)])
@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_full_jacobian_step(cams, cname, R, precision, tol):
    """One implicit step with the full-Jacobian Newton step against the
    oracle's; it reaches the root the lagged step reaches."""
    case = make_case(**CASES[cname], restriction=R, steps=1, nl_tol=1e-9, precision=precision)
    out = {}
    for jac in (0, 1):
        h, bc, keep = gpu_handle(case, jacobian=jac)
        try:
            p = case.inp["p0"].copy()
            out[jac] = (p, cams.cams_solve(h, p.copy(), case.inp["dt"], bc, p))
        finally:
            cams.cams_destroy(h)
    case.opt.full_jacobian = True
    q, sto = oracle.run(case.pb, case.opt, case.inp["p0"], case.inp["dt"], 1)
    p, st = out[1]
    assert st.converged and sto[0].converged
    assert _rel(p, q) < tol
    assert abs(st.newton_its - sto[0].newton_its) <= 1
    # the lagged step's pressure: the same root, each side stopped at
    # ||eps|| < 1e-9 ||eps_0||, which leaves them about 1e-7 apart
    assert _rel(p, out[0][0]) < 1e-6
