"""Test Case 1 of Sec. 4.3.1 on the GPU against the oracle: scaled-down
copies (24^3 cells, coarse 8^3) of permeability Set 1 (patchy) and Set 4
(layered, 15 degrees) of Table 2, rho* = 1 + p*, Dirichlet west / east, over
the paper's three steps to t* = 0.4, 1 and 2 (non-uniform steps), FP64 and
mixed precision.

Tolerances: FP64 stops at a relative ||eps|| of 1e-10 and is held to the
FP64 parity bar at every step: pressure within 1e-9 relative L_inf, the
Newton count and the step's C-AMS count each within one.  Mixed precision
stops at 1e-8 and is held to the FP64 oracle's pressure within 1e-6 relative
L_inf with the Newton count within one."""
import numpy as np
import pytest

import oracle

from _cases import gpu_handle, make_case

pytestmark = pytest.mark.gpu

_ORACLE = {}


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _case(name, precision, nl_tol):
    return make_case(name, nx=24, ny=24, nz=24, nl_tol=nl_tol, precision=precision)


def _oracle(name, nl_tol):
    key = (name, nl_tol)
    if key not in _ORACLE:
        case = _case(name, 0, nl_tol)
        _ORACLE[key] = oracle.run(case.pb, case.opt, case.inp["p0"], case.inp["dts"], 3)
    return _ORACLE[key]


@pytest.mark.parametrize("name", ["3d-64x64x64-set1", "3d-64x64x64-set4"])
@pytest.mark.parametrize("precision,nl_tol,tol", [(0, 1e-10, 1e-9), (1, 1e-8, 1e-6)])
def test_three_steps_to_t_star_2(cams, name, precision, nl_tol, tol):
    case = _case(name, precision, nl_tol)
    h, bc, keep = gpu_handle(case)
    try:
        p = case.inp["p0"].copy()
        stats = []
        for d in case.inp["dts"]:
            pn = p.copy()
            st = cams.cams_solve(h, pn, d, bc, p)
            stats.append((bool(st.converged), int(st.newton_its), int(st.cams_its)))
    finally:
        cams.cams_destroy(h)
    q, sto = _oracle(name, 1e-10 if precision == 0 else 1e-8)
    assert all(c for c, _, _ in stats) and all(s.converged for s in sto)
    for (c, n, its), so in zip(stats, sto):
        assert abs(n - so.newton_its) <= 1, (n, so.newton_its)
        if precision == 0:
            assert abs(its - so.cams_its) <= 1, (its, so.cams_its)
    rel = float(np.abs(p - q).max() / np.abs(q).max())
    assert rel < tol
