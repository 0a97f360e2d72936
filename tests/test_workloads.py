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


def _lag_corr(f, dz, dy, dx):
    """Empirical correlation of a (nz, ny, nx) field at a lattice lag."""
    nz, ny, nx = f.shape
    def sl(d, n):
        return (slice(0, n - d), slice(d, n)) if d >= 0 else (slice(-d, n), slice(0, n + d))
    (az, bz), (ay, by), (ax, bx) = sl(dz, nz), sl(dy, ny), sl(dx, nx)
    a, b = f[az, ay, ax], f[bz, by, bx]
    a, b = a - a.mean(), b - b.mean()
    return float((a * b).mean() / np.sqrt((a * a).mean() * (b * b).mean()))


def test_permeability_sets_of_table_2():
    """Sets 1-6: ln k variance 4 and mean -1; patchy sets isotropic with a
    spherical correlation of ~0.31 at 4 cells (range 0.125 L = 8 cells at
    64^3); layered sets correlated over ~30 cells along the axis 15 degrees
    from y (lag (dx, dy) = (-1, 4): ~0.8), short across it ((1, 4): 0) and
    vertically (range 0.64 cells: 0); three steps ending at t* = 0.4, 1, 2."""
    for k in range(1, 7):
        w = WORKLOADS[f"3d-{(64, 128, 256)[(k - 1) % 3]}x{(64, 128, 256)[(k - 1) % 3]}x"
                      f"{(64, 128, 256)[(k - 1) % 3]}-set{k}"]
        assert w.coarse == (8, 8, 8) and w.law == 1 and w.c_or_eta == 1.0
        assert w.t_stars == (0.4, 1.0, 2.0) and w.steps == 3
    p1 = make_inputs(WORKLOADS["3d-64x64x64-set1"])
    l1 = np.log(p1["kx"]).reshape(64, 64, 64)
    assert abs(l1.mean() + 1.0) < 0.3 and abs(l1.var() - 4.0) < 0.8
    c = [_lag_corr(l1, 0, 0, 4), _lag_corr(l1, 0, 4, 0), _lag_corr(l1, 4, 0, 0)]
    assert all(0.15 < v < 0.5 for v in c), c
    np.testing.assert_allclose(np.array(p1["dts"]) / p1["tau"], [0.4, 0.6, 1.0])
    p4 = make_inputs(WORKLOADS["3d-64x64x64-set4"])
    l4 = np.log(p4["kx"]).reshape(64, 64, 64)
    assert abs(l4.mean() + 1.0) < 0.5 and abs(l4.var() - 4.0) < 1.2
    along, across, vert = _lag_corr(l4, 0, 4, -1), _lag_corr(l4, 0, 4, 1), _lag_corr(l4, 1, 0, 0)
    assert along > 0.6 and abs(across) < 0.2 and abs(vert) < 0.2, (along, across, vert)


def test_non_uniform_steps_in_the_oracle():
    """A reduced Set 1 (16^3, coarse 4^3) over the three steps: oracle.run
    with the list of steps equals the steps taken one at a time, and each
    converges."""
    w = WORKLOADS["3d-64x64x64-set1"].with_(nx=16, ny=16, nz=16, coarse=(4, 4, 4))
    inp = make_inputs(w)
    g = oracle.Grid(w.nx, w.ny, w.nz, inp["dx"], inp["dy"], inp["dz"])
    pb = oracle.Problem.build(g, oracle.Fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi),
                              oracle.BC(True, w.p_west, w.p_east), inp["kx"], inp["ky"], inp["kz"])
    opt = oracle.Options(coarse=w.coarse, basis=w.basis, n_post=w.n_post, nl_tol=w.nl_tol)
    p, st = oracle.run(pb, opt, inp["p0"], inp["dts"], 3)
    assert len(st) == 3 and all(s.converged for s in st)
    q = inp["p0"]
    for d in inp["dts"]:
        q, _ = oracle.run(pb, opt, q, d, 1)
    np.testing.assert_array_equal(p, q)
    assert 0.0 <= p.min() and p.max() <= 1.0 + 1e-9
