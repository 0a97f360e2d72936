"""Engine-level GPU checks that need no oracle arithmetic: the pipelined
ILU(0) wavefronts (factorisation and both sweeps; one tile per warp or 2 x 2
tile blocks per CTA) equal the level-scheduled ones bit for bit, the
bounded device-side wait times out cleanly, a handle can be reused for a
new permeability field, and the host and device memory spaces agree."""
import os

import numpy as np
import pytest

from _cases import gpu_handle, make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _iterate(cams, case, n, mode):
    """mode: 'level' (one launch per hyperplane), 'warp' (one tile per warp,
    tile edges through L2) or 'cta' (2 x 2 tile blocks per CTA, edges inside
    a block through shared memory)."""
    env = {"CAMS_ILU_LEVEL": "1" if mode == "level" else "0",
           "CAMS_ILU_CTA": "1" if mode == "cta" else "0"}
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        h, bc, keep = gpu_handle(case)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v
    try:
        rng = np.random.default_rng(3)
        p_nu = rng.uniform(0, 1, case.N)
        p_n = rng.uniform(0, 1, case.N)
        cams.cams_assemble(h, p_nu, p_n, case.inp["dt"], bc)
        cams.cams_update_basis(h, True)
        d = cams.cams_get(h, cams.CAMS_Q_ILU_DIAG, np.zeros(case.N))
        res = cams.cams_iterate(h, n)
        p = cams.cams_get(h, cams.CAMS_Q_PRESSURE, np.zeros(case.N))
        return res, p, d
    finally:
        cams.cams_destroy(h)


@pytest.mark.parametrize("shape,coarse", [((40, 40, 1), (5, 5, 1)), ((30, 30, 20), (10, 10, 10)),
                                          ((24, 17, 13), (6, 17, 13)), ((64, 9, 33), (8, 3, 3)),
                                          ((12, 8, 6), (2, 4, 3)), ((20, 72, 40), (10, 8, 8))])
def test_pipelined_sweeps_equal_level_schedule(cams, shape, coarse):
    """Ragged tiles in y and z, 2D and 3D, a single tile and many: same
    arithmetic, same bits."""
    case = make_case("3d-200x200x100", nx=shape[0], ny=shape[1], nz=shape[2], coarse=coarse,
                     n_post=3, n_pre=1)
    r0, p0, d0 = _iterate(cams, case, 3, "level")
    for mode in ("warp", "cta"):
        r1, p1, d1 = _iterate(cams, case, 3, mode)
        assert np.array_equal(d1, d0), mode    # ILU(0) factorisation wavefront
        assert np.array_equal(p1, p0), mode    # forward/backward sweeps
        assert np.array_equal(r1, r0), mode


def test_bounded_wait_times_out_and_context_survives(cams):
    case = make_case("2d-40x40", nx=20, ny=20, steps=1)
    h, bc, keep = gpu_handle(case)
    try:
        code = cams.cams_selftest_wait(h)
        assert code == cams.CAMS_ETIMEOUT
        assert "wait" in cams.cams_last_error(h)
        # the context is still usable
        p = case.inp["p0"].copy()
        st = cams.cams_solve(h, case.inp["p0"], case.inp["dt"], bc, p)
        assert st.converged
    finally:
        cams.cams_destroy(h)


def test_set_permeability_matches_fresh_handle(cams):
    a = make_case("3d-200x200x100", nx=20, ny=20, nz=10, coarse=(5, 5, 5), seed=0)
    b = make_case("3d-200x200x100", nx=20, ny=20, nz=10, coarse=(5, 5, 5), seed=1)
    h, bc, keep = gpu_handle(a)
    try:
        pa = a.inp["p0"].copy()
        cams.cams_solve(h, a.inp["p0"], a.inp["dt"], bc, pa)
        cams.cams_set_permeability(h, b.inp["kx"], b.inp["ky"], b.inp["kz"])
        pb = b.inp["p0"].copy()
        st = cams.cams_solve(h, b.inp["p0"], b.inp["dt"], bc, pb)
    finally:
        cams.cams_destroy(h)
    h2, bc2, keep2 = gpu_handle(b)
    try:
        q = b.inp["p0"].copy()
        st2 = cams.cams_solve(h2, b.inp["p0"], b.inp["dt"], bc2, q)
    finally:
        cams.cams_destroy(h2)
    assert np.array_equal(pb, q)
    assert st.basis_rebuilt == st2.basis_rebuilt


def test_device_memspace_matches_host(cams):
    torch = pytest.importorskip("torch")
    case = make_case("3d-100x100x50-wells", nx=20, ny=20, nz=10, coarse=(5, 5, 5), steps=1)
    h, bc, keep = gpu_handle(case)
    try:
        p = case.inp["p0"].copy()
        cams.cams_solve(h, case.inp["p0"], case.inp["dt"], bc, p)
    finally:
        cams.cams_destroy(h)
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(np.ascontiguousarray(case.inp[k])).to(dev) for k in ("kx", "ky", "kz", "p0")}
    sc = torch.from_numpy(case.inp["src_cell"].astype(np.int32)).to(dev)
    sr = torch.from_numpy(case.inp["src_rate"]).to(dev)
    w, inp = case.w, case.inp
    grid = cams.cams_grid(w.nx, w.ny, w.nz, inp["dx"], inp["dy"], inp["dz"])
    fluid = cams.cams_fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi)
    opt = cams.make_options(w.coarse, basis=w.basis, restriction=w.restriction, n_post=w.n_post,
                            nl_tol=w.nl_tol, adapt_theta=w.adapt_theta, memspace=cams.CAMS_DEVICE)
    hd = cams.cams_setup(grid, fluid, opt, t["kx"], t["ky"], t["kz"])
    try:
        cams.cams_set_stream(hd, torch.cuda.current_stream(dev).cuda_stream)
        bcd, keepd = cams.make_bc(False, 0.0, 0.0, sc, sr)
        pd = t["p0"].clone()
        cams.cams_solve(hd, t["p0"], inp["dt"], bcd, pd)
        torch.cuda.synchronize()
    finally:
        cams.cams_destroy(hd)
    assert np.array_equal(pd.cpu().numpy(), p)


def test_schedule_switch_on_a_live_handle(cams):
    """cams_set_schedule on a handle that has already iterated (and captured
    its iteration graph): every accepted ILU(0) tile schedule continues from
    the same state with the same bits, since the schedules share the per-cell
    arithmetic; the coarse-solve schedules sum in different orders, so their
    iterates agree to rounding.  A refused schedule leaves the handle's
    schedule unchanged."""
    case = make_case("3d-200x200x100", nx=40, ny=40, nz=20, coarse=(10, 10, 10), n_post=3)
    h, bc, keep = gpu_handle(case)
    try:
        rng = np.random.default_rng(5)
        p_nu = rng.uniform(0, 1, case.N)
        cams.cams_assemble(h, p_nu, p_nu, case.inp["dt"], bc)
        cams.cams_update_basis(h, True)
        runs = {}
        for ilu in (0, 1):
            for cl in (0, 1):
                try:
                    cams.cams_set_schedule(h, ilu, cl)
                except cams.CamsError:
                    assert cams.cams_get_schedule(h) != (ilu, cl)
                    continue
                assert cams.cams_get_schedule(h) == (ilu, cl)
                cams.cams_assemble(h, p_nu, p_nu, case.inp["dt"], bc)
                res = cams.cams_iterate(h, 3)
                p = cams.cams_get(h, cams.CAMS_Q_PRESSURE, np.zeros(case.N))
                runs[(ilu, cl)] = (res, p)
        assert runs
        for cl in (0, 1):
            if (0, cl) in runs and (1, cl) in runs:
                assert np.array_equal(runs[(0, cl)][0], runs[(1, cl)][0])
                assert np.array_equal(runs[(0, cl)][1], runs[(1, cl)][1])
        ps = [p for _, p in runs.values()]
        for p in ps[1:]:
            assert np.abs(p - ps[0]).max() <= 1e-12 * np.abs(ps[0]).max()
        # a refused value leaves the schedule as it was
        before = cams.cams_get_schedule(h)
        with pytest.raises(cams.CamsError):
            cams.cams_set_schedule(h, 2, 0)
        assert cams.cams_get_schedule(h) == before
    finally:
        cams.cams_destroy(h)
