"""Write the golden record of the 3D wells workload at full size from the oracle.

The workload is the 100 x 100 x 50 layered field (ln k standard deviation 3,
correlation lengths 0.2 / 0.2 / 0.02 of the domain, kz = 0.1 k), c dp = 0.2,
an injector and a producer as vertical line wells in opposite corners
(Reading R16), 10 implicit steps, 10 x 10 x 5 coarse blocks, the (B1) basis
with adaptive updates at theta = 0.1 (Sec. 4.1.2), 5 ILU(0) post-smoothing
steps, MSFE or MSFV restriction (Sec. 3, Eq. 7), relative stopping test
NL_TOL per step (1e-5 unless GOLDEN_NL_TOL says otherwise).  (The
workload's 1e-6 is out of reach at full size: in the second step the
oracle's lagged-density linearisations stall near 1.5e-6 relative, its inner
loops falling to 3 or 4 iterations, and 50 of them do not meet it; in the
third step they stall above 1e-4.  The record keeps the converged steps and
the first one that does not converge.)
For every step the record holds the oracle's Newton and C-AMS counts (per
linearisation), the number of local entities rebuilt, convergence, the 2-norm,
maximum, minimum and sum of the pressure field, and the pressure at a fixed
seeded sample of cells (plus the perforated cells and the eight corners).

Only the oracle and the seeded input generator are called; nothing here comes
from the GPU path.  Run from the repository root:

    python tests/golden/make_wells_golden.py [msfe|msfv ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle.solver import BasisState, solve_step  # noqa: E402
from oracle.wirebasket import build_wirebasket  # noqa: E402
from workloads import WORKLOADS, make_inputs  # noqa: E402

WORKLOAD = "3d-100x100x50-wells"
SEED = 0
N_SAMPLE = 256
NL_TOL = float(os.environ.get("GOLDEN_NL_TOL", "1e-5"))


def golden_path(restriction: int) -> str:
    return os.path.join(HERE, f"wells_100x100x50_seed{SEED}_{('msfe', 'msfv')[restriction]}"
                              f"_tol{NL_TOL:g}.json")


def sample_cells(w, inp) -> np.ndarray:
    """Seeded sample of cells, the perforated cells and the eight corners."""
    N = w.nx * w.ny * w.nz
    rng = np.random.default_rng(20170517)
    cells = set(rng.choice(N, N_SAMPLE, replace=False).tolist())
    cells |= set(int(c) for c in inp["src_cell"])
    for z in (0, w.nz - 1):
        for y in (0, w.ny - 1):
            for x in (0, w.nx - 1):
                cells.add(x + w.nx * (y + w.ny * z))
    return np.array(sorted(cells), dtype=np.int64)


def make(restriction: int) -> dict:
    w = WORKLOADS[WORKLOAD].with_(restriction=restriction, nl_tol=NL_TOL)
    inp = make_inputs(w, SEED)
    g = oracle.Grid(w.nx, w.ny, w.nz, inp["dx"], inp["dy"], inp["dz"])
    bc = oracle.BC(inp["dirichlet"], w.p_west, w.p_east, inp["src_cell"], inp["src_rate"],
                   inp["fix_cell"], inp["fix_value"])
    pb = oracle.Problem.build(g, oracle.Fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi), bc,
                              inp["kx"], inp["ky"], inp["kz"])
    opt = oracle.Options(coarse=w.coarse, basis=w.basis, restriction=w.restriction,
                         n_pre=w.n_pre, n_post=w.n_post, lin_rtol=w.lin_rtol, nl_tol=w.nl_tol,
                         adapt_theta=w.adapt_theta, max_newton=w.max_newton,
                         max_cams=w.max_cams)
    wb = build_wirebasket(g, opt.coarse)
    state = BasisState(wb)
    cells = sample_cells(w, inp)
    p = inp["p0"].copy()
    steps = []
    for k, dt in enumerate(inp["dts"]):
        t0 = time.time()
        p, st = solve_step(pb, wb, state, opt, p, dt)
        steps.append({
            "newton_its": st.newton_its, "cams_its": st.cams_its,
            "cams_per_newton": list(st.cams_per_newton), "basis_rebuilt": st.basis_rebuilt,
            "converged": bool(st.converged),
            "eps_rel_final": float(st.eps_hist[-1] / st.eps_hist[0]),
            "eps_hist": [float(v) for v in st.eps_hist],
            "p_norm2": float(np.linalg.norm(p)), "p_max": float(p.max()),
            "p_min": float(p.min()), "p_sum": float(p.sum()),
            "p_sample": [float(v) for v in p[cells]],
        })
        print(f"{('MSFE', 'MSFV')[restriction]} step {k}: {st.newton_its} Newton, "
              f"{st.cams_its} C-AMS, {st.basis_rebuilt} rebuilt, converged {st.converged} "
              f"({time.time() - t0:.0f} s)", flush=True)
        if not st.converged:
            break
    return {
        "workload": WORKLOAD, "seed": SEED,
        "restriction": ("MSFE", "MSFV")[restriction],
        "grid": [w.nx, w.ny, w.nz], "coarse": list(w.coarse), "basis": w.basis,
        "adapt_theta": w.adapt_theta, "n_post": w.n_post, "nl_tol": w.nl_tol,
        "lin_rtol": w.lin_rtol, "max_cams": w.max_cams, "max_newton": w.max_newton,
        "sample_cells": [int(c) for c in cells],
        "source": "oracle/ (tests/golden/make_wells_golden.py); Sec. 4.1.2 adaptive updates, "
                  "Table 1 iteration, Sec. 4.1.1 stopping tests",
        "steps": steps,
    }


def main(argv):
    which = argv or ["msfe", "msfv"]
    for name in which:
        r = {"msfe": 0, "msfv": 1}[name]
        rec = make(r)
        with open(golden_path(r), "w") as f:
            json.dump(rec, f, indent=0)
        print("wrote", golden_path(r), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
