"""The no-allocation residual entry point against the engine's own residual.

cams_residual_norm_noalloc exists for callers that cannot call cudaMalloc
(code under CUDA-graph capture, frameworks that own all device memory,
time-critical loops).  It keeps its reduction scratch in a static device
array, so this test also checks that a second call in a row, which finds the
first call's partial sums still in that array, gives the same answer.  The
file name sorts last so a run that stops at the first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from _cases import gpu_handle, make_case

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_engine_twice():
    torch = pytest.importorskip("torch")
    from paper_1705_05783_gb300 import cams
    case = make_case("3d-100x100x50-wells", nx=40, ny=30, nz=20, coarse=(10, 10, 5))
    N = case.N
    rng = np.random.default_rng(11)
    p_nu = rng.uniform(-0.5, 1.0, N)
    p_n = rng.uniform(-0.5, 1.0, N)
    h, bc, keep = gpu_handle(case)
    try:
        cams.cams_assemble(h, p_nu, p_n, case.inp["dt"], bc)
        A = cams.cams_get(h, cams.CAMS_Q_MATRIX, np.zeros(4 * N))
        f = cams.cams_get(h, cams.CAMS_Q_RHS, np.zeros(N))
        r_ref = cams.cams_get(h, cams.CAMS_Q_RESIDUAL, np.zeros(N))
        cams.cams_update_basis(h, True)
        norm_ref = cams.cams_iterate(h, 0)[0]      # the engine's ||f - A p|| at p = p_nu
    finally:
        cams.cams_destroy(h)
    dev = torch.device("cuda", 0)
    dA = torch.from_numpy(A).to(dev)
    df = torch.from_numpy(f).to(dev)
    dp = torch.from_numpy(p_nu).to(dev)
    parts = [dA[k * N:(k + 1) * N] for k in range(4)]
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):
        r = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        code, norm = cams.cams_residual_norm_noalloc(case.w.nx, case.w.ny, case.w.nz, *parts,
                                                     df, dp, r, stream)
        assert code == cams.CAMS_OK, cams.cams_last_error()
        rr = r.cpu().numpy()
        # same per-cell arithmetic; the norm sums in a different block order
        np.testing.assert_allclose(rr, r_ref, rtol=0, atol=1e-13 * np.abs(r_ref).max())
        assert abs(norm - norm_ref) <= 1e-13 * norm_ref
        assert abs(norm - np.linalg.norm(r_ref)) <= 1e-12 * norm_ref


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1705_05783_gb300 import cams
    fake = 1 << 20            # never dereferenced: the size check comes first
    code, _ = cams.cams_residual_norm_noalloc(1024, 1024, 1024, fake, fake, fake, fake, fake,
                                              fake, None)
    assert code == cams.CAMS_EINVAL
    msg = cams.cams_last_error()
    assert "268435456" in msg and "1073741824" in msg
