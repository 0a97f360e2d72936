"""The paper-shape sets of Test Case 1 at 256^3 (Sec. 4.3.1, Table 2, Sets 3
and 6) with both coarsenings the paper uses there (8^3 and 16^3 blocks,
Sec. 4.1.5), and the two engine paths they need:

- 16^3 blocks: a 15^3 interior's banded local system (3375 unknowns,
  half-bandwidth 225) exceeds shared memory, so the blocked local solver
  keeps its window in global memory;
- 8^3 blocks at 256^3: the coarse system has 32,768 unknowns (half-bandwidth
  1,057) and its band substitution keeps its vectors in global memory.

At sizes the oracle solves in seconds the two paths are held to it (basis
values, a whole step with its counts); at 256^3 a step is checked by
properties that hold at any size: it converges, its pressure is a root of
the oracle's nonlinear residual (Eq. 19) to the stopping tolerance, and it
obeys the discrete maximum principle of the Dirichlet 1 / 0 problem."""
import numpy as np
import pytest

import oracle
from oracle.basis import basis_operator, prolongation
from oracle.problem import epsilon
from oracle.wirebasket import build_wirebasket

from _cases import gpu_handle, make_case, p_from_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("precision", [0, 1])
def test_global_window_local_solver_matches_oracle(cams, precision):
    """16^3 blocks on a 32^3 patchy field: the 15^3 interiors go through the
    global-memory window.  P against the oracle's staged basis within
    eps * max cond(M_e) of the working precision (as for the shared-memory
    solver)."""
    case = make_case("3d-64x64x64-set1", nx=32, ny=32, nz=32, coarse=(16, 16, 16),
                     precision=precision)
    h, bc, keep = gpu_handle(case)
    try:
        p0 = case.inp["p0"]
        cams.cams_assemble(h, p0, p0, case.inp["dts"][0], bc)
        cams.cams_update_basis(h, True)
        wb = build_wirebasket(case.pb.grid, case.w.coarse)
        Pg, vals, cols = p_from_gpu(h, case.N, wb.Nc)
    finally:
        cams.cams_destroy(h)
    lin = oracle.assemble(case.pb, p0, p0, case.inp["dts"][0])
    Ab = basis_operator(case.pb, 4, lin.rho, lin.c, p0, case.inp["dts"][0])
    Po = prolongation(Ab, wb).to_csr(wb.Nc)
    err = float(np.abs((Pg - Po).toarray()).max())
    from test_gpu_parity import p_tolerance    # eps(float64) * max cond(M_e)
    tol = p_tolerance(Ab, wb)
    if precision:
        tol *= np.finfo(np.float32).eps / np.finfo(np.float64).eps
    print(f"[global-window P, precision {precision}] max |dP| = {err:.2e}, bound {tol:.2e}")
    assert err < tol


def test_large_blocks_step_matches_oracle(cams):
    """One step of the 32^3 field with 16^3 blocks in FP64 at 1e-10, held to
    the FP64 parity bar: pressure within 1e-9, Newton and C-AMS counts
    within one."""
    case = make_case("3d-64x64x64-set1", nx=32, ny=32, nz=32, coarse=(16, 16, 16), nl_tol=1e-10)
    h, bc, keep = gpu_handle(case)
    try:
        p = case.inp["p0"].copy()
        st = cams.cams_solve(h, case.inp["p0"].copy(), case.inp["dts"][0], bc, p)
    finally:
        cams.cams_destroy(h)
    q, sto = oracle.run(case.pb, case.opt, case.inp["p0"], case.inp["dts"][0], 1)
    assert st.converged and sto[0].converged
    assert _rel(p, q) < 1e-9
    assert abs(st.newton_its - sto[0].newton_its) <= 1
    assert abs(st.cams_its - sto[0].cams_its) <= 1


@pytest.mark.parametrize("name,coarse", [("3d-256x256x256-set3", (8, 8, 8)),
                                         ("3d-256x256x256-set3", (16, 16, 16)),
                                         ("3d-256x256x256-set6", (16, 16, 16))])
def test_paper_shape_256_first_step(cams, name, coarse):
    """The first step (t* = 0 -> 0.4) of a 256^3 set, mixed precision, at the
    paper's tolerance: converged, a root of the oracle's Eq. 19 residual to
    that tolerance (twice it, for the summation order of 16.7M terms), and
    0 <= p <= 1."""
    case = make_case(name, coarse=coarse, precision=1)
    h, bc, keep = gpu_handle(case)
    try:
        p = case.inp["p0"].copy()
        st = cams.cams_solve(h, case.inp["p0"].copy(), case.inp["dts"][0], bc, p)
    finally:
        cams.cams_destroy(h)
    assert st.converged
    e0 = np.linalg.norm(epsilon(case.pb, case.inp["p0"], case.inp["p0"], case.inp["dts"][0]))
    e1 = np.linalg.norm(epsilon(case.pb, p, case.inp["p0"], case.inp["dts"][0]))
    print(f"[{name} {coarse}] {st.newton_its} Newton, {st.cams_its} C-AMS, "
          f"||eps|| {e1 / e0:.2e} of the start")
    assert e1 <= 2 * case.w.nl_tol * e0
    assert p.min() >= -1e-9 and p.max() <= 1 + 1e-9
