"""The mixed preconditioner's coarse solve (Eq. 15's coarse problem
R A P p_c = R r, Sec. 3) by the inverse factor: the FP32 band LDL^T of the
Galerkin matrix, Z = L^{-1} formed once per factorisation, and each solve
p_c = Z^T D^{-1} Z R r.  In exact arithmetic this is the substitution;
in FP32 it differs from it by rounding only.

Held to the FP64 oracle's C-AMS iterates (Table 1 steps 4-7) on coarse
systems of several 32-row blocks with a ragged last one, beside the FP32
substitution with the FP64 factor's copy (CAMS_COARSE_INV=0) as a control:
the two FP32 coarse solves must track the oracle equally well."""
import os

import numpy as np
import pytest

import oracle
from _cases import gpu_handle, make_case
from oracle.basis import basis_operator, prolongation
from oracle.coarse import coarse_factor, coarse_operator, restriction
from oracle.ilu import ilu0
from oracle.solver import cams_iteration
from oracle.wirebasket import build_wirebasket

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _iterates(cams, case, inv, n):
    old = os.environ.get("CAMS_COARSE_INV")
    os.environ["CAMS_COARSE_INV"] = "1" if inv else "0"
    try:
        h, bc, keep = gpu_handle(case)
    finally:
        if old is None:
            del os.environ["CAMS_COARSE_INV"]
        else:
            os.environ["CAMS_COARSE_INV"] = old
    try:
        p0 = case.inp["p0"]
        cams.cams_assemble(h, p0, p0, case.inp["dts"][0], bc)
        cams.cams_update_basis(h, True)
        out = []
        for _ in range(n):
            res = cams.cams_iterate(h, 1)
            out.append((cams.cams_get(h, cams.CAMS_Q_PRESSURE, np.zeros(case.N)), float(res[-1])))
    finally:
        cams.cams_destroy(h)
    return out


@pytest.mark.parametrize("kw", [
    dict(nx=40, ny=40, nz=20, coarse=(4, 4, 4)),     # 500 coarse nodes, half-width 57
    dict(nx=36, ny=28, nz=20, coarse=(4, 4, 5)),     # 252 coarse nodes, ragged block
])
def test_inverse_factor_iterates_track_the_oracle(cams, kw):
    case = make_case("3d-200x200x100-mixed", **kw)
    n = 4
    p0 = case.inp["p0"]
    dt = case.inp["dts"][0]
    lin = oracle.assemble(case.pb, p0, p0, dt)
    wb = build_wirebasket(case.pb.grid, case.w.coarse)
    Ab = basis_operator(case.pb, case.w.basis, lin.rho, lin.c, p0, dt)
    P = prolongation(Ab, wb).to_csr(wb.Nc)
    R = restriction(0, P, wb)
    lu = coarse_factor(coarse_operator(R, lin.A, P))
    LU = ilu0(lin.A)
    p = p0.copy()
    ref = []
    for _ in range(n):
        p = cams_iteration(lin.A, lin.f, p, P, R, lu, LU, case.w.n_pre, case.w.n_post)
        ref.append((p.copy(), float(np.linalg.norm(lin.f - lin.A @ p))))
    for inv in (True, False):
        got = _iterates(cams, case, inv, n)
        for k, ((pg, rg), (po, ro)) in enumerate(zip(got, ref)):
            ep, er = _rel(pg, po), abs(rg - ro) / ro
            print(f"[{'inverse' if inv else 'substitution'} {kw['coarse']}] iterate {k + 1}: "
                  f"|dp| {ep:.2e}, residual {er:.2e}")
            # FP32 preconditioner: each iterate within FP32 rounding of the
            # FP64 one, amplified by the coarse system's conditioning
            assert ep < 1e-4, (inv, k, ep)
            assert er < 1e-2, (inv, k, er)
