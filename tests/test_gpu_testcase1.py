"""Test Case 1 of Sec. 4.3.1 on the GPU against the oracle: scaled-down
copies (24^3 cells, coarse 8^3) of permeability Set 1 (patchy) and Set 4
(layered, 15 degrees) of Table 2, rho* = 1 + p*, Dirichlet west / east, over
the paper's three steps to t* = 0.4, 1 and 2 (non-uniform steps), FP64 and
mixed precision.

Tolerances: converged pressures (relative 1e-8 on ||eps||) within 1e-7
relative L_inf in FP64 and 1e-6 in mixed precision after the third step (two
iterates that both meet the stopping test differ by up to that much once an
inner count differs by one), Newton counts within one per step."""
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


def _case(name, precision):
    return make_case(name, nx=24, ny=24, nz=24, nl_tol=1e-8, precision=precision)


def _oracle(name):
    if name not in _ORACLE:
        case = _case(name, 0)
        _ORACLE[name] = oracle.run(case.pb, case.opt, case.inp["p0"], case.inp["dts"], 3)
    return _ORACLE[name]


@pytest.mark.parametrize("name", ["3d-64x64x64-set1", "3d-64x64x64-set4"])
@pytest.mark.parametrize("precision,tol", [(0, 1e-7), (1, 1e-6)])
def test_three_steps_to_t_star_2(cams, name, precision, tol):
    case = _case(name, precision)
    h, bc, keep = gpu_handle(case)
    try:
        p = case.inp["p0"].copy()
        stats = []
        for d in case.inp["dts"]:
            pn = p.copy()
            st = cams.cams_solve(h, pn, d, bc, p)
            stats.append((bool(st.converged), int(st.newton_its)))
    finally:
        cams.cams_destroy(h)
    q, sto = _oracle(name)
    assert all(c for c, _ in stats) and all(s.converged for s in sto)
    for (c, n), so in zip(stats, sto):
        assert abs(n - so.newton_its) <= 1
    rel = float(np.abs(p - q).max() / np.abs(q).max())
    assert rel < tol
