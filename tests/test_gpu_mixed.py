"""Mixed precision (CAMS_PREC_MIXED): the multiscale preconditioner (basis
solves and P, restriction/prolongation, the coarse factor and solve (by
the inverse factor where it is small enough), ILU(0) factor and sweeps) in
FP32 inside FP64 iterative refinement; assembly, the Galerkin sums, the
residual and the update stay FP64.  The iteration's fixed point is the
FP64 one, so the converged pressure is held to the FP64 oracle: within
1e-6 relative L-infinity at a 1e-8 relative nonlinear tolerance (and much
closer in practice), with the Newton count of the oracle to within one.
The C-AMS count may grow (the preconditioner is rounded), and is bounded."""
import numpy as np
import pytest

import oracle
from _cases import gpu_handle, make_case
from oracle.basis import PRows, entity_system, prolongation
from oracle.wirebasket import build_wirebasket
from oracle.basis import basis_operator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _rel(a, b):
    s = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / s)


def _solve(cams, case, steps):
    h, bc, keep = gpu_handle(case)
    try:
        p = case.inp["p0"].copy()
        stats = []
        for _ in range(steps):
            pn = p.copy()
            st = cams.cams_solve(h, pn, case.inp["dt"], bc, p)
            stats.append((st.newton_its, st.cams_its, st.converged))
    finally:
        cams.cams_destroy(h)
    return p, stats


@pytest.mark.parametrize("cname,kw,steps", [
    ("2d-40x40", dict(nl_tol=1e-8), 3),
    ("3d-200x200x100", dict(nx=30, ny=30, nz=20, nl_tol=1e-8), 1),
    ("3d-100x100x50-wells", dict(nx=40, ny=40, nz=20, nl_tol=1e-8, max_cams=60), 1),
])
def test_mixed_solve_matches_fp64_oracle(cams, cname, kw, steps):
    case = make_case(cname, precision=1, steps=steps, **kw)
    p, stats = _solve(cams, case, steps)
    q, sto = oracle.run(case.pb, case.opt, case.inp["p0"], case.inp["dt"], steps)
    assert _rel(p, q) < 1e-6
    for (n, c, conv), so in zip(stats, sto):
        assert conv
        assert abs(n - so.newton_its) <= 1
        assert c <= 2 * so.cams_its + 2 * n


@pytest.mark.parametrize("cname,kw", [("2d-40x40", {}),
                                      ("3d-200x200x100", dict(nx=30, ny=30, nz=20)),
                                      ("3d-100x100x50-wells", dict(nx=40, ny=40, nz=20, basis=1))])
def test_mixed_basis_close_to_oracle(cams, cname, kw):
    """FP32 local solves: both sides are backward stable, so the basis values
    differ by about 64 * eps(float32) * the largest local condition number."""
    case = make_case(cname, precision=1, **kw)
    h, bc, keep = gpu_handle(case)
    try:
        p0 = case.inp["p0"]
        cams.cams_assemble(h, p0, p0, case.inp["dt"], bc)
        cams.cams_update_basis(h, True)
        N = case.N
        G = np.zeros(8 * N)
        J = np.zeros(8 * N, dtype=np.int32)
        cams.cams_get(h, cams.CAMS_Q_PROLONG, G)
        cams.cams_get_int(h, cams.CAMS_Q_PROLONG_J, J)
        G, J = G.reshape(8, N), J.reshape(8, N)
    finally:
        cams.cams_destroy(h)
    wb = build_wirebasket(case.pb.grid, case.w.coarse)
    lin = oracle.assemble(case.pb, p0, p0, case.inp["dt"])
    Ab = basis_operator(case.pb, case.w.basis, lin.rho, lin.c, p0, case.inp["dt"])
    P = prolongation(Ab, wb).to_csr(wb.Nc).toarray()
    Pg = np.zeros_like(P)
    for s in range(8):
        ok = J[s] >= 0
        Pg[np.arange(N)[ok], J[s][ok]] += G[s][ok]
    kmax = 1.0
    Pr = PRows(wb.grid.N)
    for e in wb.entities:
        M, _ = entity_system(Ab, wb, Pr, e)
        if M.shape[0] > 1:
            kmax = max(kmax, np.linalg.cond(M))
    tol = 64 * np.finfo(np.float32).eps * kmax
    assert np.abs(Pg - P).max() < tol


def test_mixed_pipelined_sweeps_equal_level_schedule(cams):
    """The FP32 wavefronts: pipelined (CTA blocks or warp tiles) and
    level-scheduled give the same bits."""
    import os
    case = make_case("3d-200x200x100", nx=20, ny=72, nz=40, coarse=(10, 8, 8), n_post=3,
                     precision=1)
    out = []
    for level, cta in ((False, "1"), (False, "0"), (True, "0")):
        env = {"CAMS_ILU_LEVEL": "1" if level else "0", "CAMS_ILU_CTA": cta}
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
            res = cams.cams_iterate(h, 3)
            p = cams.cams_get(h, cams.CAMS_Q_PRESSURE, np.zeros(case.N))
            out.append((d, p, res))
        finally:
            cams.cams_destroy(h)
    d0, p0, r0 = out[-1]
    for d1, p1, r1 in out[:-1]:
        assert np.array_equal(d1, d0)
        assert np.array_equal(p1, p0)
        assert np.array_equal(r1, r0)


def test_mixed_full_size_matches_fp64_engine(cams):
    """The 4M-cell step in mixed precision against the FP64 engine (which the
    parity tests hold to the oracle): a property that holds at any size."""
    res = {}
    for prec in (0, 1):
        case = make_case("3d-200x200x100", precision=prec)
        p, stats = _solve(cams, case, 1)
        res[prec] = (p, stats[0])
    (p64, (n64, c64, ok64)), (p32, (n32, c32, ok32)) = res[0], res[1]
    assert ok64 and ok32
    assert _rel(p32, p64) < 1e-6
    assert abs(n32 - n64) <= 1
    assert c32 <= 2 * c64
