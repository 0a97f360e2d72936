"""Training of the learned basis surrogate on the GPU.

The network (4 layers of 3x3x3 convolutions, see cams.h) is trained on basis
functions that the method itself computes, by default in the energy norm of
the interior error (the norm a basis function's error costs the coarse space;
a masked MSE is the alternative): for seeded permeability fields the
engine builds the basis with its exact local solves, cams_surrogate_data cuts
every full dual-block interior's patch into network inputs and targets, and
the library's own layer kernels (cams_net_conv_forward/backward, cams_net_mse,
cams_net_adam) run the forward pass, the backward pass and the Adam updates.
PyTorch only holds the device memory.

    python -m paper_1705_05783_gb300.surrogate --out params.npy
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

from . import cams

LAYERS = [(cams.CAMS_NET_IN, cams.CAMS_NET_HID), (cams.CAMS_NET_HID, cams.CAMS_NET_HID),
          (cams.CAMS_NET_HID, cams.CAMS_NET_HID), (cams.CAMS_NET_HID, cams.CAMS_NET_OUT)]
PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "surrogate_params.npy")


def offsets():
    """(w offset, b offset) of every layer in the parameter vector."""
    out, o = [], 0
    for ci, co in LAYERS:
        out.append((o, o + co * ci * 27))
        o += co * ci * 27 + co
    assert o == cams.CAMS_NET_PARAMS
    return out


def init_params(seed=0):
    """He-uniform weights (fan-in 27 ci), zero biases, float32."""
    rng = np.random.default_rng(seed)
    p = np.zeros(cams.CAMS_NET_PARAMS, np.float32)
    for (ci, co), (ow, ob) in zip(LAYERS, offsets()):
        lim = np.sqrt(6.0 / (27 * ci))
        p[ow:ob] = rng.uniform(-lim, lim, co * ci * 27).astype(np.float32)
    return p


def load_params(path=PARAMS_FILE):
    return np.load(path).astype(np.float32)


class Trainer:
    """Parameters, gradients, Adam moments and activation buffers for
    batches of B patches of edge S, all on the GPU."""

    def __init__(self, params, B, S, device, lr=1e-3, loss="energy"):
        import torch
        self.torch = torch
        self.B, self.S, self.lr, self.kind = B, S, lr, loss
        f32 = dict(dtype=torch.float32, device=device)
        self.p = torch.from_numpy(np.asarray(params, np.float32)).to(device)
        self.g = torch.zeros_like(self.p)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        S3 = S ** 3
        self.acts = [None] + [torch.zeros((B, co, S3), **f32) for _, co in LAYERS]
        self.gbuf = [torch.zeros((B, cams.CAMS_NET_HID, S3), **f32) for _ in range(2)]
        self.gy = torch.zeros((B, cams.CAMS_NET_OUT, S3), **f32)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.scratch = torch.zeros(512, dtype=torch.float64, device=device)
        self.t = 0
        self.off = offsets()

    def _w(self, k, buf):
        ow, ob = self.off[k]
        ci, co = LAYERS[k]
        return buf[ow:ob], buf[ob:ob + co]

    def forward(self, x, B=None):
        B = B or self.B
        a = x
        for k, (ci, co) in enumerate(LAYERS):
            w, b = self._w(k, self.p)
            out = self.acts[k + 1]
            cams.cams_net_conv_forward(B, self.S, ci, co, a, w, b, int(k < len(LAYERS) - 1), out)
            a = out
        self.acts[0] = x
        return a

    def step(self, x, target, mask):
        """One Adam step on the masked MSE of the batch; returns the loss
        as a device tensor."""
        self.gradients(x, target, mask)
        self.t += 1
        cams.cams_net_adam(self.p.numel(), self.p, self.g, self.m, self.v, self.lr, 0.9, 0.999,
                           1e-8, self.t)
        return self.loss

    def gradients(self, x, target, mask):
        """Loss (device) and its gradient with respect to every parameter
        (self.g, in the parameter layout) for one batch."""
        y = self.forward(x)
        self.loss_of(y, x, target, mask)
        g = self.gy
        for k in range(len(LAYERS) - 1, -1, -1):
            ci, co = LAYERS[k]
            w, _ = self._w(k, self.p)
            gw, gb = self._w(k, self.g)
            gx = self.gbuf[k % 2] if k > 0 else None
            xact = self.acts[k] if k > 0 else None
            cams.cams_net_conv_backward(self.B, self.S, ci, co, self.acts[k], w, g, xact,
                                        None if gx is None else gx[:, :ci], gw, gb)
            g = gx[:, :ci] if gx is not None else None
        return self.loss

    def loss_of(self, y, x, target, mask, kind=None):
        """The batch loss into self.loss and its gradient into self.gy:
        the energy norm of the interior error (default) or the masked MSE."""
        count = max(float(mask.sum().item()), 1.0)
        if (kind or self.kind) == "energy":
            cams.cams_net_energy(y.shape[0], self.S, cams.CAMS_NET_OUT, cams.CAMS_NET_IN, y, target,
                                 mask, x, count, self.gy, self.loss, self.scratch)
        else:
            cams.cams_net_mse(y.numel(), y, target, mask, count, self.gy, self.loss, self.scratch)
        return self.loss

    def params(self):
        return self.p.cpu().numpy().copy()


def training_fields(n=20, seed=100):
    """Seeded fields of the 4M-cell layout (200x200x100, coarse 10^3) with
    sigma drawn uniformly in [1, 4]; seeds distinct from the workloads'."""
    from workloads import WORKLOADS
    rng = np.random.default_rng(seed)
    base = WORKLOADS["3d-200x200x100"]
    return [base.with_(sigma=float(rng.uniform(1.0, 4.0)), seeds=(seed + k,), precision=0)
            for k in range(n)]


def generate(fields, device, max_per_field=100000):
    """Patches (x, target, mask) of every full interior of every field."""
    import torch
    from workloads import make_inputs
    xs, ts, ms = [], [], []
    for w in fields:
        inp = make_inputs(w)
        grid = cams.cams_grid(w.nx, w.ny, w.nz, inp["dx"], inp["dy"], inp["dz"])
        fluid = cams.cams_fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi)
        opt = cams.make_options(w.coarse, basis=w.basis, restriction=w.restriction,
                                n_post=w.n_post, nl_tol=w.nl_tol, precision=0)
        h = cams.cams_setup(grid, fluid, opt, inp["kx"], inp["ky"], inp["kz"])
        try:
            bc, keep = cams.make_bc(inp["dirichlet"], w.p_west, w.p_east)
            cams.cams_assemble(h, inp["p0"], inp["p0"], inp["dt"], bc)
            cams.cams_update_basis(h, True)
            S3 = (w.coarse[0] + 1) ** 3
            n_all = cams.cams_surrogate_data(h, 0)
            n_take = min(max_per_field, max(n_all, 1))
            x = torch.zeros((n_take, cams.CAMS_NET_IN, S3), dtype=torch.float32, device=device)
            t = torch.zeros((n_take, cams.CAMS_NET_OUT, S3), dtype=torch.float32, device=device)
            m = torch.zeros_like(t)
            got = cams.cams_surrogate_data(h, n_take, x, t, m)
            xs.append(x[:got]); ts.append(t[:got]); ms.append(m[:got])
        finally:
            cams.cams_destroy(h)
    return torch.cat(xs), torch.cat(ts), torch.cat(ms)


def train(x, t, m, S, steps=3000, batch=64, lr=1e-3, seed=0, log=None, val=None, loss="energy"):
    """Adam on shuffled batches; the learning rate halves at 50% and 75% of
    the steps.  Returns (params, [(step, train loss, val loss)])."""
    import torch
    device = x.device
    tr = Trainer(init_params(seed), batch, S, device, lr, loss)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    hist = []
    perm = torch.randperm(n, generator=gen)
    pos = 0
    for s in range(1, steps + 1):
        if s in (steps // 2, (3 * steps) // 4):
            tr.lr *= 0.5
        if pos + batch > n:
            perm = torch.randperm(n, generator=gen)
            pos = 0
        idx = perm[pos:pos + batch].to(device)
        pos += batch
        loss = tr.step(x[idx].contiguous(), t[idx].contiguous(), m[idx].contiguous())
        if s == 1 or s % 250 == 0 or s == steps:
            vl = evaluate(tr, *val, kind=tr.kind) if val is not None else None
            hist.append((s, float(loss.item()), vl))
            if log:
                log(f"step {s} loss {hist[-1][1]:.4e} val {vl}")
    return tr.params(), hist


def evaluate(tr, x, t, m, kind="mse"):
    """Masked MSE (or the energy loss) of the current parameters over a data
    set (whole batches)."""
    tot, cnt = 0.0, 0.0
    for p0 in range(0, x.shape[0] - tr.B + 1, tr.B):
        xb = x[p0:p0 + tr.B].contiguous()
        y = tr.forward(xb)
        mb = m[p0:p0 + tr.B].contiguous()
        c = float(mb.sum().item())
        tr.loss_of(y, xb, t[p0:p0 + tr.B].contiguous(), mb, kind)
        tot += float(tr.loss.item()) * c
        cnt += c
    return tot / max(cnt, 1.0)


def time_network(B, S=11, repeats=10):
    """CUDA-event time of one forward pass of the network over B patches of
    S^3 voxels: the tensor-core entry point (BF16 operands, FP32
    accumulation) and the FP32 CUDA-core layer kernels, with random
    parameters.  Returns {name: ms}."""
    import torch
    dev = torch.device("cuda", 0)
    params = init_params(5)
    p = torch.from_numpy(params).to(dev)
    x = torch.randn(B, cams.CAMS_NET_IN, S ** 3, device=dev)
    y = torch.zeros(B, cams.CAMS_NET_OUT, S ** 3, device=dev)
    nb = cams.cams_net_tc_work_bytes(B, S)
    work = torch.zeros(nb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def tc():
        code = cams.cams_net_forward_tc(B, S, x, p, y, work, nb, stream)
        if code != cams.CAMS_OK:
            raise cams.CamsError(code, cams.cams_last_error())

    tr = Trainer(params, B, S, dev)
    out = {}
    for name, fn, n in (("tensor_core", tc, repeats), ("fp32_cuda_core", lambda: tr.forward(x, B), 3)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / n
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--time", type=int, default=0,
                    help="only time one forward pass over this many patches and exit")
    ap.add_argument("--out", default=PARAMS_FILE)
    ap.add_argument("--fields", type=int, default=20)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--loss", default="energy", choices=["energy", "mse"])
    a = ap.parse_args(argv)
    if a.time > 0:
        S = 11
        flop = 2.0 * a.time * S ** 3 * 27 * sum(ci * co for ci, co in LAYERS)
        for name, ms in time_network(a.time, S).items():
            print(f"{name}: {ms:.3f} ms for {a.time} patches of {S}^3, "
                  f"{flop / ms / 1e9:.1f} useful TFLOP/s", flush=True)
        return
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    device = torch.device("cuda", 0)
    t0 = time.time()
    fields = training_fields(a.fields)
    x, t, m = generate(fields[:-1], device)
    xv, tv, mv = generate(fields[-1:], device)
    print(f"data: {x.shape[0]} training patches, {xv.shape[0]} validation, "
          f"{time.time() - t0:.1f} s", flush=True)
    S = round(x.shape[2] ** (1.0 / 3.0))
    t1 = time.time()
    params, hist = train(x, t, m, S, a.steps, a.batch, a.lr, val=(xv, tv, mv),
                         log=lambda s: print(s, flush=True), loss=a.loss)
    print(f"training: {time.time() - t1:.1f} s", flush=True)
    np.save(a.out, params)
    print(f"saved {a.out}", flush=True)


if __name__ == "__main__":
    main()
