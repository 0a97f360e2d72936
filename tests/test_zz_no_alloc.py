"""The no-allocation residual entry point, against the oracle and the engine.

cams_residual_norm_noalloc serves callers that cannot call cudaMalloc:
frameworks that give all device memory to their own pool, and time-critical
loops that cannot take the device-wide synchronisation of an allocation.  Its
reduction scratch is a static device array shared by every call, so the test
makes two calls in a row on different grids: the second (smaller) grid reads
fewer partial-sum slots than the first wrote, and a slot left over from the
first call would change its norm.  The file name sorts last so a run that
stops at the first failure has already run every other test; it also passes
alone in a fresh process.
"""
import numpy as np
import pytest

import oracle

from _cases import gpu_handle, make_case

pytestmark = pytest.mark.gpu


def _layout(A, w):
    """The oracle's CSR matrix in the CAMS_Q_MATRIX layout: diagonal, then
    a_{i,i-1}, a_{i,i-nx}, a_{i,i-nx*ny} stored at cell i (0 where absent)."""
    N = w.nx * w.ny * w.nz
    i = np.arange(N)
    out = [A.diagonal().copy()]
    for off, ok in ((1, i % w.nx > 0), (w.nx, (i // w.nx) % w.ny > 0),
                    (w.nx * w.ny, i // (w.nx * w.ny) > 0)):
        a = np.zeros(N)
        a[ok] = np.asarray(A[i[ok], i[ok] - off]).ravel()
        out.append(a)
    return out


def _call(cams, torch, w, parts, f, p, want_r=True, want_norm=True):
    dev = torch.device("cuda", 0)
    d = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (*parts, f, p)]
    r = torch.full((w.nx * w.ny * w.nz,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    code, norm = cams.cams_residual_norm_noalloc(w.nx, w.ny, w.nz, *d, r if want_r else None,
                                                 stream, want_norm=want_norm)
    assert code == cams.CAMS_OK, cams.cams_last_error()
    return r.cpu().numpy(), norm


def test_noalloc_residual_matches_oracle_and_engine_twice():
    torch = pytest.importorskip("torch")
    from paper_1705_05783_gb300 import cams

    big = make_case("3d-100x100x50-wells", nx=40, ny=30, nz=20, coarse=(10, 10, 5))
    small = make_case("3d-200x200x100", nx=20, ny=10, nz=10, coarse=(10, 10, 10))
    for case, seed in ((big, 11), (small, 12)):       # 3 partial sums, then 1
        N = case.N
        rng = np.random.default_rng(seed)
        p_nu = rng.uniform(-0.5, 1.0, N)
        p_n = rng.uniform(-0.5, 1.0, N)
        # the oracle's system and its residual f - A p
        lin = oracle.assemble(case.pb, p_nu, p_n, case.inp["dt"])
        r_or = lin.f - lin.A @ p_nu
        r, norm = _call(cams, torch, case.w, _layout(lin.A, case.w), lin.f, p_nu)
        scale = np.abs(r_or).max()
        # same per-cell products, summed in another order: a few ulps of the terms
        terms = np.abs(lin.f) + abs(lin.A) @ np.abs(p_nu)
        assert np.all(np.abs(r - r_or) <= 64 * np.finfo(float).eps * terms)
        assert abs(norm - np.linalg.norm(r_or)) <= 1e-12 * np.linalg.norm(r_or)
        # the engine's own residual entry point on the engine's matrix
        h, bc, keep = gpu_handle(case)
        try:
            cams.cams_assemble(h, p_nu, p_n, case.inp["dt"], bc)
            A = cams.cams_get(h, cams.CAMS_Q_MATRIX, np.zeros(4 * N))
            f = cams.cams_get(h, cams.CAMS_Q_RHS, np.zeros(N))
            r_eng = cams.cams_get(h, cams.CAMS_Q_RESIDUAL, np.zeros(N))
            cams.cams_update_basis(h, True)
            norm_eng = cams.cams_iterate(h, 0)[0]    # the engine's ||f - A p|| at p = p_nu
        finally:
            cams.cams_destroy(h)
        parts = [A[k * N:(k + 1) * N] for k in range(4)]
        r2, norm2 = _call(cams, torch, case.w, parts, f, p_nu)
        np.testing.assert_allclose(r2, r_eng, rtol=0, atol=1e-13 * scale)
        assert abs(norm2 - norm_eng) <= 1e-13 * norm_eng
        # norm only (r = NULL) and residual only (norm_out = NULL)
        _, norm3 = _call(cams, torch, case.w, parts, f, p_nu, want_r=False)
        assert norm3 == norm2
        r4, none = _call(cams, torch, case.w, parts, f, p_nu, want_norm=False)
        assert none is None and np.array_equal(r4, r2)


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1705_05783_gb300 import cams
    fake = 1 << 20            # never dereferenced: the size check comes first
    code, _ = cams.cams_residual_norm_noalloc(1024, 1024, 1024, fake, fake, fake, fake, fake,
                                              fake, None)
    assert code == cams.CAMS_EINVAL
    msg = cams.cams_last_error()
    assert "268435456" in msg and "1073741824" in msg
