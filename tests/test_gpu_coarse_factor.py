"""The coarse-system factorisation (Sec. 3: the coarse problem R A P p_c =
R r of Eq. 15 solved directly) read back from the engine and held to its
definition: R A P = L D L^T with L unit lower triangular inside the band
and D > 0, for the FP64 engine and for the mixed one (whose coarse
factorisation stays FP64).

Two pins that do not use the engine's own arithmetic: the product L D L^T
reproduces the engine's R A P in the band order within the componentwise
backward-error bound of a Cholesky-type factorisation (|dA| <= g |L| D |L|^T
with g = (m + 2) u, Higham Thm. 10.3 in LDL^T form), and the factor
agrees with LAPACK's Cholesky factor C of the same matrix (l = C / diag C,
d = diag(C)^2) to the forward error the matrix's conditioning allows.
Cases: several 16-column blocks with a ragged last one, half-widths above
and below the block width, and a coarse system smaller than one block."""
import numpy as np
import pytest

from _cases import coarse_from_gpu, gpu_handle, make_case

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _factor(cams, case):
    h, bc, keep = gpu_handle(case)
    try:
        p0 = case.inp["p0"]
        cams.cams_assemble(h, p0, p0, case.inp["dts"][0], bc)
        cams.cams_update_basis(h, True)
        sizes = cams.cams_get_int(h, cams.CAMS_Q_SIZES, np.zeros(8, np.int32))
        Nc, nc = int(sizes[1]), [int(v) for v in sizes[2:5]]
        Ac, _ = coarse_from_gpu(h, nc)
        order = cams.cams_get_int(h, cams.CAMS_Q_COARSE_ORDER, np.zeros(Nc + 1, np.int32))
        m = int(order[0])
        band = cams.cams_get(h, cams.CAMS_Q_COARSE_FACTOR, np.zeros(Nc * (m + 1)))
    finally:
        cams.cams_destroy(h)
    pos = order[1:]
    assert sorted(pos.tolist()) == list(range(Nc))
    A = np.zeros((Nc, Nc))
    A[np.ix_(pos, pos)] = Ac                       # A[pos[I], pos[J]] = Ac[I, J]
    L = np.eye(Nc)
    d = np.zeros(Nc)
    for q in range(Nc):
        col = band[q * (m + 1):(q + 1) * (m + 1)]
        d[q] = col[0]
        hi = min(q + m, Nc - 1)
        L[q + 1:hi + 1, q] = col[1:hi - q + 1]
    return A, L, d, m


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kw", [
    dict(nx=40, ny=40, nz=20, coarse=(4, 4, 4)),     # 500 coarse nodes, half-width 57
    dict(nx=36, ny=28, nz=20, coarse=(4, 4, 5)),     # 252 coarse nodes, half-width 33
    dict(nx=48, ny=16, nz=8, coarse=(4, 4, 4)),      # 12 x 4 x 2 = 96 nodes, half-width 11
    dict(nx=16, ny=16, nz=16, coarse=(8, 8, 8)),     # 2 x 2 x 2 = 8 nodes (one partial block)
])
def test_coarse_factor_reproduces_rap(cams, kw, prec):
    case = make_case("3d-200x200x100", precision=prec, **kw)
    A, L, d, m = _factor(cams, case)
    Nc = A.shape[0]
    # band structure of the ordering: nothing of A lies outside the half-width
    i, j = np.nonzero(A)
    assert np.abs(i - j).max() <= m
    assert np.all(d > 0), "R A P is SPD for MSFE of a symmetric A"
    LD = L * d
    got = LD @ L.T
    bound = (m + 2) * EPS * (np.abs(L) * d) @ np.abs(L).T
    excess = np.abs(got - A) - 2.0 * bound
    print(f"[{kw['coarse']} prec {prec}] Nc {Nc} m {m}: max |LDL^T - A| / bound "
          f"{float(np.max(np.abs(got - A) / np.maximum(bound, 1e-300))):.3f}")
    assert excess.max() <= 0.0, float(excess.max())
    # against LAPACK's Cholesky factor of the same matrix
    C = np.linalg.cholesky(A)
    dc = np.diag(C)
    L_ref, d_ref = C / dc, dc ** 2
    cond = np.linalg.cond(A)
    tol = 64 * EPS * cond
    el = float(np.abs(L - L_ref).max() / max(np.abs(L_ref).max(), 1e-300))
    ed = float(np.abs(d - d_ref).max() / d_ref.max())
    print(f"    cond {cond:.2e}: |dL| {el:.2e}, |dd| {ed:.2e} (tolerance {tol:.2e})")
    assert el <= tol and ed <= tol
