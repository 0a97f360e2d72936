"""The learned basis surrogate on the GPU.

Layer kernels against the float64 oracle of the network (oracle/net.py):
forward values and gradients to 1e-5 relative (FP32 arithmetic, sums of a
few hundred terms).  A whole-network gradient from the library's kernels
against the oracle's backward pass.  Training on patches the engine
generates lowers the loss.  In the engine: with the trained parameters a
solve still reaches the oracle's pressure (the surrogate only changes the
preconditioner), the residual gate hands the rejected interiors to the exact
solve, and on an unseen field the trained network predicts the interior
basis values with less than half the energy-norm error of the multilinear
baseline alone (the network with all-zero parameters) and lower gate ratios."""
import os

import numpy as np
import pytest

import oracle
from oracle.net import adam_step, conv_backward, conv_forward, mse, network_backward, network_forward
from _cases import gpu_handle, make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1705_05783_gb300 import cams, surrogate
    return torch, cams, surrogate


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("relu", [0, 1])
def test_conv_forward_backward_match_oracle(env, relu):
    torch, cams, _ = env
    rng = np.random.default_rng(5)
    B, ci, co, S = 3, 11, 10, 6
    x = rng.standard_normal((B, ci, S, S, S))
    w = 0.3 * rng.standard_normal((co, ci, 27))
    b = rng.standard_normal(co)
    xd, wd, bd = _dev(torch, x), _dev(torch, w), _dev(torch, b)
    y = torch.zeros((B, co, S, S, S), device="cuda")
    cams.cams_net_conv_forward(B, S, ci, co, xd, wd, bd, relu, y)
    torch.cuda.synchronize()
    xr = x.astype(np.float32).astype(np.float64)
    wr = w.astype(np.float32).astype(np.float64)
    br = b.astype(np.float32).astype(np.float64)
    assert _rel(y.cpu().numpy(), conv_forward(xr, wr, br, bool(relu))) < 1e-5
    gy = rng.standard_normal((B, co, S, S, S))
    xact = rng.standard_normal((B, ci, S, S, S))            # the ReLU mask's source
    gx = torch.zeros_like(xd)
    gw = torch.zeros_like(wd)
    gb = torch.zeros_like(bd)
    cams.cams_net_conv_backward(B, S, ci, co, xd, wd, _dev(torch, gy), _dev(torch, xact), gx, gw, gb)
    torch.cuda.synchronize()
    gyr = gy.astype(np.float32).astype(np.float64)
    rx, rw, rb = conv_backward(xr, wr, gyr)
    rx = rx * (xact.astype(np.float32) > 0)
    assert _rel(gx.cpu().numpy(), rx) < 1e-5
    assert _rel(gw.cpu().numpy(), rw) < 1e-5
    assert _rel(gb.cpu().numpy(), rb) < 1e-5


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as the tensor-core
    kernels round their operands; returned in float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _tc_work(torch, cams, B, S):
    n = cams.cams_net_tc_work_bytes(B, S)
    return torch.zeros(n, dtype=torch.uint8, device="cuda"), n


@pytest.mark.parametrize("S,ci,co,relu", [(11, 12, 32, 1), (11, 32, 32, 1), (11, 32, 8, 0),
                                          (6, 5, 13, 1), (4, 32, 16, 0)])
def test_tensor_core_conv_matches_oracle(env, S, ci, co, relu):
    """One 3x3x3 layer on the tensor cores (BF16 operands, FP32 accumulation
    in tensor memory) against the oracle's convolution of the same
    BF16-rounded input and weights: only the FP32 accumulation order differs,
    so every output is within 1e-4 of the sum of the magnitudes of its (at
    most 27 x 32 = 864) terms, the worst-case FP32 rounding of such a sum.
    Ragged channel counts and small patches exercise the zero padding of
    channels, tiles and borders."""
    torch, cams, _ = env
    rng = np.random.default_rng(11 + S + ci)
    B = 5
    x = rng.standard_normal((B, ci, S, S, S))
    w = 0.3 * rng.standard_normal((co, ci, 27))
    b = rng.standard_normal(co)
    y = torch.full((B, co, S, S, S), float("nan"), device="cuda")
    work, nbytes = _tc_work(torch, cams, B, S)
    code = cams.cams_net_conv_forward_tc(B, S, ci, co, _dev(torch, x), _dev(torch, w), _dev(torch, b),
                                         relu, y, work, nbytes)
    assert code == cams.CAMS_OK, cams.cams_last_error()
    yg = y.cpu().numpy().astype(np.float64)
    xb, wb, br = bf16(x), bf16(w), b.astype(np.float32).astype(np.float64)
    ref = conv_forward(xb, wb, br, bool(relu))
    mag = conv_forward(np.abs(xb), np.abs(wb), np.abs(br), False)
    assert np.all(np.isfinite(yg))
    err = np.abs(yg - ref)
    print(f"[tc conv S={S} {ci}->{co}] max |dy| / magnitude = {(err / mag).max():.2e}")
    assert np.all(err <= 1e-4 * mag)


def test_tensor_core_network_matches_oracle(env):
    """The whole 4-layer network on the tensor cores against the oracle's
    network with the kernels' precision applied between layers (input,
    weights and every hidden activation rounded to BF16, FP32 output).  A
    hidden value within FP32 rounding of a BF16 rounding boundary may round
    the other way on the GPU, a one-ulp (2^-8 relative) change of one input
    of the next layer, so the bar is 1e-3 of the output's magnitude sum."""
    torch, cams, surrogate = env
    rng = np.random.default_rng(12)
    B, S = 4, 11
    params = surrogate.init_params(5)
    x = rng.standard_normal((B, cams.CAMS_NET_IN, S, S, S))
    y = torch.full((B, cams.CAMS_NET_OUT, S, S, S), float("nan"), device="cuda")
    work, nbytes = _tc_work(torch, cams, B, S)
    code = cams.cams_net_forward_tc(B, S, _dev(torch, x), _dev(torch, params), y, work, nbytes)
    assert code == cams.CAMS_OK, cams.cams_last_error()
    a = bf16(x)
    amag = np.abs(a)
    L = surrogate.LAYERS
    for k, ((ci, co), (ow, ob)) in enumerate(zip(L, surrogate.offsets())):
        w = params[ow:ob].astype(np.float64).reshape(co, ci, 27)
        b = params[ob:ob + co].astype(np.float64)
        last = k == len(L) - 1
        a = conv_forward(a, bf16(w), b, not last)
        amag = conv_forward(amag, np.abs(bf16(w)), np.abs(b), False)
        if not last:
            a = bf16(a)
    yg = y.cpu().numpy().astype(np.float64)
    err = np.abs(yg - a)
    print(f"[tc network] max |dy| / magnitude = {(err / amag).max():.2e}")
    assert np.all(err <= 1e-3 * amag)


def test_tensor_core_workspace_is_checked(env):
    torch, cams, _ = env
    work = torch.zeros(16, dtype=torch.uint8, device="cuda")
    x = torch.zeros((1, 4, 5, 5, 5), device="cuda")
    code = cams.cams_net_conv_forward_tc(1, 5, 4, 4, x, torch.zeros(4 * 4 * 27, device="cuda"),
                                         torch.zeros(4, device="cuda"), 0, x, work, 16)
    assert code == cams.CAMS_EINVAL and "workspace" in cams.cams_last_error()


def test_mse_and_adam_match_oracle(env):
    torch, cams, _ = env
    rng = np.random.default_rng(6)
    n = 5000
    p, t = rng.standard_normal(n), rng.standard_normal(n)
    m = (rng.random(n) < 0.5).astype(np.float64)
    grad = torch.zeros(n, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    scratch = torch.zeros(512, dtype=torch.float64, device="cuda")
    cams.cams_net_mse(n, _dev(torch, p), _dev(torch, t), _dev(torch, m), m.sum(), grad, loss, scratch)
    torch.cuda.synchronize()
    pr, tr = p.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64)
    L, G = mse(pr, tr, m, m.sum())
    assert abs(loss.item() - L) < 1e-6 * L
    assert _rel(grad.cpu().numpy(), G) < 1e-5
    par, g = _dev(torch, p), _dev(torch, t)
    mm, vv = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    P, M, V = pr.copy(), np.zeros(n), np.zeros(n)
    for step in (1, 2, 3):
        cams.cams_net_adam(n, par, g, mm, vv, 1e-2, 0.9, 0.999, 1e-8, step)
        P, M, V = adam_step(P, tr, M, V, 1e-2, 0.9, 0.999, 1e-8, step)
    torch.cuda.synchronize()
    assert np.abs(par.cpu().numpy() - P).max() < 1e-5


def test_energy_loss_matches_oracle(env):
    torch, cams, _ = env
    from oracle.net import energy_loss
    rng = np.random.default_rng(8)
    B, C, S, cx = 3, 8, 6, 12
    x = rng.standard_normal((B, cx, S, S, S))
    t = rng.standard_normal((B, C, S, S, S))
    p = t + 0.2 * rng.standard_normal(t.shape)
    m = np.zeros_like(t); m[:, :, 1:-1, 1:-1, 1:-1] = 1.0
    grad = torch.zeros((B, C, S, S, S), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    scratch = torch.zeros(512, dtype=torch.float64, device="cuda")
    cams.cams_net_energy(B, S, C, cx, _dev(torch, p), _dev(torch, t), _dev(torch, m), _dev(torch, x),
                         m.sum(), grad, loss, scratch)
    torch.cuda.synchronize()
    f = lambda a: a.astype(np.float32).astype(np.float64)
    E, G = energy_loss(f(p), f(t), m, f(x)[:, :3])
    assert abs(loss.item() - E) < 1e-5 * E
    assert _rel(grad.cpu().numpy(), G) < 1e-5


def test_network_gradient_matches_oracle(env):
    """Whole 4-layer network: the library's forward and backward kernels
    against the oracle's, same parameters and data."""
    torch, cams, surrogate = env
    rng = np.random.default_rng(7)
    B, S = 2, 7
    params = surrogate.init_params(3)
    tr = surrogate.Trainer(params, B, S, torch.device("cuda"), loss="mse")
    x = rng.standard_normal((B, cams.CAMS_NET_IN, S ** 3))
    t = 0.1 * rng.standard_normal((B, cams.CAMS_NET_OUT, S ** 3))
    m = (rng.random((B, cams.CAMS_NET_OUT, S ** 3)) < 0.7).astype(np.float64)
    loss = tr.gradients(_dev(torch, x), _dev(torch, t), _dev(torch, m))
    torch.cuda.synchronize()
    g = tr.g.cpu().numpy().astype(np.float64)
    layers = []
    for (ci, co), (ow, ob) in zip(surrogate.LAYERS, surrogate.offsets()):
        layers.append((params[ow:ob].astype(np.float64).reshape(co, ci, 27),
                       params[ob:ob + co].astype(np.float64)))
    shp = (B, -1, S, S, S)
    xr = x.astype(np.float32).astype(np.float64).reshape(shp)
    y, acts = network_forward(xr, layers)
    L, gy = mse(y, t.astype(np.float32).reshape(shp), m.reshape(shp), m.sum())
    assert abs(float(loss.item()) - L) < 1e-4 * L
    ref = network_backward(acts, layers, gy)
    for (gw, gb), (ow, ob) in zip(ref, surrogate.offsets()):
        assert _rel(g[ow:ob], gw.ravel()) < 1e-4
        assert _rel(g[ob:ob + gb.size], gb) < 1e-4


def test_training_on_engine_patches_lowers_the_loss(env):
    torch, cams, surrogate = env
    fields = [f.with_(nx=60, ny=60, nz=40) for f in surrogate.training_fields(3)]
    x, t, m = surrogate.generate(fields, torch.device("cuda"))
    assert x.shape[0] == 3 * 5 * 5 * 3                      # full interiors of 6x6x4 coarse cells
    # targets: exact basis values minus the multilinear baseline, mask = interior
    assert float(m.sum().item()) == x.shape[0] * 8 * 9 ** 3
    params, hist = surrogate.train(x, t, m, 11, steps=300, batch=16, lr=2e-3, loss="energy")
    first, last = hist[0][1], hist[-1][1]
    assert np.isfinite(last) and last < 0.5 * first


def _params_or_skip(surrogate):
    if not os.path.exists(surrogate.PARAMS_FILE):
        pytest.skip("no trained surrogate parameters")
    return surrogate.load_params()


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_surrogate_solve_matches_oracle(env, precision, tol):
    """With the trained surrogate the step still converges to the oracle's
    pressure; some interiors come from the network, the rest from the exact
    solve."""
    torch, cams, surrogate = env
    params = _params_or_skip(surrogate)
    case = make_case("3d-200x200x100", nx=60, ny=60, nz=40, nl_tol=1e-8, precision=precision)
    h, bc, keep = gpu_handle(case)
    try:
        cams.cams_set_surrogate(h, params, 0.3)
        p = case.inp["p0"].copy()
        st = cams.cams_solve(h, case.inp["p0"].copy(), case.inp["dt"], bc, p)
        sizes = cams.cams_get_int(h, cams.CAMS_Q_SIZES, np.zeros(8, np.int32))
    finally:
        cams.cams_destroy(h)
    q, sto = oracle.run(case.pb, case.opt, case.inp["p0"], case.inp["dt"], 1)
    assert st.converged
    assert _rel(p, q) < tol
    assert abs(st.newton_its - sto[0].newton_its) <= 1
    assert 0 <= sizes[7] <= 75


def test_trained_network_gains_over_the_baseline(env):
    """On a field it was not trained on: the trained network's error in the
    interior basis values (energy norm) is well below the multilinear
    baseline's (the all-zero network), its gate ratios are lower, and with it the step
    still converges to the exact-basis pressure (at a 1e-10 nonlinear
    tolerance: a different P takes a different path to the tolerance)."""
    torch, cams, surrogate = env
    params = _params_or_skip(surrogate)
    zero = np.zeros_like(params)
    case = make_case("3d-200x200x100", nx=100, ny=100, nz=60, nl_tol=1e-10, precision=1)
    # prediction error against the exact basis
    h, bc, keep = gpu_handle(case.__class__(case.w.with_(precision=0), case.inp, case.pb, case.opt))
    try:
        cams.cams_assemble(h, case.inp["p0"], case.inp["p0"], case.inp["dt"], bc)
        cams.cams_update_basis(h, True)
        n = cams.cams_surrogate_data(h, 0)
        S3 = 11 ** 3
        x = torch.zeros((n, cams.CAMS_NET_IN, S3), device="cuda")
        t = torch.zeros((n, cams.CAMS_NET_OUT, S3), device="cuda")
        m = torch.zeros_like(t)
        assert cams.cams_surrogate_data(h, n, x, t, m) == n == 9 * 9 * 5
    finally:
        cams.cams_destroy(h)
    err = {}
    for name, pr in (("trained", params), ("baseline", zero)):
        tr = surrogate.Trainer(pr, 5, 11, torch.device("cuda"))
        err[name] = surrogate.evaluate(tr, x, t, m, kind="energy")
    # gate ratios and the solve
    out = {}
    for name, pr in (("trained", params), ("baseline", zero), ("exact", None)):
        h, bc, keep = gpu_handle(case)
        try:
            if pr is not None:
                cams.cams_set_surrogate(h, pr, 1.0)
            p = case.inp["p0"].copy()
            st = cams.cams_solve(h, case.inp["p0"].copy(), case.inp["dt"], bc, p)
            ratio = None
            if pr is not None:
                ratio = cams.cams_get(h, cams.CAMS_Q_SURR_RATIO, np.zeros(n))
            out[name] = (st.cams_its, st.converged, p, ratio)
        finally:
            cams.cams_destroy(h)
    print("\ninterior MSE", err, "median gate ratio",
          {k: float(np.median(v[3])) for k, v in out.items() if v[3] is not None},
          "C-AMS its", {k: v[0] for k, v in out.items()})
    assert err["trained"] < 0.5 * err["baseline"]          # energy norm of the interior error
    assert np.median(out["trained"][3]) < np.median(out["baseline"][3])
    assert out["trained"][1] and out["baseline"][1]
    assert _rel(out["trained"][2], out["exact"][2]) < 1e-6
