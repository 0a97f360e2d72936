"""Host-side checks of the synthetic workloads (no GPU): the prescribed
columns of Test Case 2 sit where the paper puts them and on no coarse node,
the stretched grids keep the stated aspect ratio and time scale, and the
ensemble's members are seeded, divisible by their coarse blocks and within
the stated size range."""
import numpy as np

import oracle
from workloads import WORKLOADS, ensemble_members, line_columns, make_inputs


def test_test_case_2_columns_and_stretching():
    for a in (1, 5, 10):
        w = WORKLOADS[f"3d-64x64x64-lines-a{a}"]
        cells, vals = line_columns(w)
        x, y, z = cells % w.nx, (cells // w.nx) % w.ny, cells // (w.nx * w.ny)
        assert set(zip(x[vals == 1.0], y[vals == 1.0])) == {(0, 0)}
        assert set(zip(x[vals == 0.0], y[vals == 0.0])) == {(63, 63)}
        assert sorted(z[vals == 1.0]) == list(range(64))
        wb = oracle.build_wirebasket(oracle.Grid(w.nx, w.ny, w.nz, 1.0, 1.0, 1.0), w.coarse)
        assert np.all(wb.level[cells] > 0)                 # never a coarse node
        inp = make_inputs(w)
        assert np.isclose(inp["dx"] / inp["dy"], a) and inp["dy"] == inp["dz"]
        # the time scale uses alpha L as the length
        assert np.isclose(inp["tau"], w.mu * w.phi * a ** 2 / inp["k_bar"])


def test_ensemble_members():
    m1, m2 = ensemble_members(64), ensemble_members(64)
    assert [w.name for w in m1] == [w.name for w in m2]
    assert len({w.seeds[0] for w in m1}) == 64
    for w in m1:
        assert 32 ** 3 <= w.n_cells <= 128 * 128 * 64
        assert all(n % b == 0 for n, b in zip((w.nx, w.ny, w.nz), w.coarse))
        assert 1.0 <= w.sigma <= 4.0 and w.precision == 1
    assert len({(w.nx, w.ny, w.nz) for w in m1}) > 4      # uneven sizes
