"""Workload definitions: grids, coarsening, fluid, boundary conditions, time
step and solver options of the synthetic cases, and the recipe that turns
one into concrete input arrays.

Non-dimensionalisation follows Sec. 4 of the paper: h = 1/nx, cells of
h x h x h (stretched to alpha h x h x h when the aspect ratio alpha != 1, so
the domain is alpha L long in x with L = 1), Delta p = p_west - p_east = 1,
mu = 1, phi = 0.1, and the time step is Delta t = Delta t* . tau with
tau = mu phi (alpha L)^2 / (K_bar Delta p), K_bar the geometric mean of k
(Sec. 4; Test Case 2 of Sec. 4.2.2 takes alpha L as the length scale).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

from .fields import lognormal_permeability


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    coarse: tuple            # primal block size (bx, by, bz)
    sigma: float             # standard deviation of ln k
    corr: tuple              # correlation lengths / L along (x, y, z)
    kz_ratio: float = 1.0
    cov: str = "exponential"
    angle_deg: float = 0.0
    law: int = 0             # 0: rho = rho0 exp(c p); 1: rho = rho0 (1 + eta p)
    c_or_eta: float = 0.1
    rho0: float = 1.0
    mu: float = 1.0
    phi: float = 0.1
    bc: str = "dirichlet_we"  # or "wells", or "lines" (two prescribed vertical columns)
    p_west: float = 1.0
    p_east: float = 0.0
    well_rate: float = 0.02   # drawdown scale of the well rates (wells only)
    steps: int = 1
    dt_star: float = 0.01
    basis: int = 4            # 1..4 = Eqs. (B1)..(B4)
    restriction: int = 0      # 0 = MSFE, 1 = MSFV
    n_pre: int = 0
    n_post: int = 1
    lin_rtol: float = 0.1
    nl_tol: float = 1e-6
    adapt_theta: float = 0.1
    max_newton: int = 50
    max_cams: int = 200
    precision: int = 0        # engine option: 0 = FP64, 1 = FP32 preconditioner in FP64 refinement
    alpha: float = 1.0        # grid aspect ratio: dx / alpha = dy = dz
    seeds: tuple = (0,)
    lnk_mean: float = 0.0     # mean of ln k
    t_stars: tuple = ()       # end times t* of the steps (non-uniform steps); () = steps x dt_star

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz

    def with_(self, **kw):
        return replace(self, **kw)


WORKLOADS = {
    # 2D 40x40 unit square, 8x8 coarse, exponential rho with c dp = 0.1,
    # Dirichlet west/east, 5 steps of dt* = 0.01, (B4), MSFE, 1 ILU(0) post step.
    "2d-40x40": Workload(
        name="2d-40x40", nx=40, ny=40, nz=1, coarse=(5, 5, 1), sigma=2.0,
        corr=(0.1, 0.1, 0.1), c_or_eta=0.1, steps=5, basis=4, restriction=0,
        n_post=1, nl_tol=1e-6, seeds=tuple(range(20))),
    # 3D 100x100x50 layered field, kz = 0.1 k, c dp = 0.2, two wells in
    # opposite corners, 10 steps, 10x10x5 coarse, (B1) adaptive at 0.1.
    "3d-100x100x50-wells": Workload(
        name="3d-100x100x50-wells", nx=100, ny=100, nz=50, coarse=(10, 10, 5),
        sigma=3.0, corr=(0.2, 0.2, 0.02), kz_ratio=0.1, c_or_eta=0.2,
        bc="wells", steps=10, basis=1, restriction=0, n_post=5,
        nl_tol=1e-6, adapt_theta=0.1, seeds=(0, 1, 2, 3, 4)),
    # 3D 200x200x100 (4M cells), sigma 3, corr 0.1 L, 20x20x10 coarse,
    # Dirichlet west/east, (B4), MSFE, 5 ILU(0) post steps, tolerance 1e-8.
    "3d-200x200x100": Workload(
        name="3d-200x200x100", nx=200, ny=200, nz=100, coarse=(10, 10, 10),
        sigma=3.0, corr=(0.1, 0.1, 0.1), c_or_eta=0.1, steps=1, basis=4,
        restriction=0, n_post=5, nl_tol=1e-8, seeds=(0,)),
    # The same problem with the multiscale preconditioner in FP32 (basis
    # solves, P, ILU(0) smoother) inside FP64 iterative refinement; FP64
    # residual, update and coarse factorisation.
    "3d-200x200x100-mixed": Workload(
        name="3d-200x200x100-mixed", nx=200, ny=200, nz=100, coarse=(10, 10, 10),
        sigma=3.0, corr=(0.1, 0.1, 0.1), c_or_eta=0.1, steps=1, basis=4,
        restriction=0, n_post=5, nl_tol=1e-8, seeds=(0,), precision=1),
}

# Test Case 2 of Sec. 4.2.2: the 64^3 patchy set (spherical variogram, ln k
# variance 4, correlation length 0.125 L in every direction), rho* = 1 + p*
# (eta = 1), pressure prescribed at the centres of the vertical columns
# (0, 0, z) = 1 and (63, 63, z) = 0 with no-flow faces, grid aspect ratio
# alpha in {1, 5, 10}, the first time step t* = 0 -> 0.4, (B4), MSFE,
# 5 ILU(0) post steps, coarsening 8x8x8 (alpha 1) and 2x8x8 (alpha 5, 10).
for _a, _cb in ((1, (8, 8, 8)), (5, (2, 8, 8)), (10, (2, 8, 8))):
    _n = f"3d-64x64x64-lines-a{_a}"
    WORKLOADS[_n] = Workload(
        name=_n, nx=64, ny=64, nz=64, coarse=_cb, sigma=2.0, corr=(0.125, 0.125, 0.125),
        cov="spherical", law=1, c_or_eta=1.0, bc="lines", steps=1, dt_star=0.4, basis=4,
        restriction=0, n_post=5, nl_tol=1e-6, alpha=float(_a), seeds=tuple(range(20)))


# Test Case 1 of Sec. 4.3.1: permeability Sets 1-6 of Table 2 (ln k variance 4,
# mean -1, spherical variogram; Sets 1-3 patchy with correlation lengths
# 0.125 L, Sets 4-6 layered with (0.5, 0.03, 0.01 or 0.06) L and the longest
# axis at 15 degrees from y), rho* = 1 + p* (eta = 1), Dirichlet 1 / 0 on the
# west / east faces, three consecutive steps to t* = 0.4, 1 and 2, (B4), MSFE,
# 5 ILU(0) post steps, coarsening 8^3.
for _k, _n, _corr, _ang in ((1, 64, (0.125, 0.125, 0.125), 0.0),
                            (2, 128, (0.125, 0.125, 0.125), 0.0),
                            (3, 256, (0.125, 0.125, 0.125), 0.0),
                            (4, 64, (0.03, 0.5, 0.01), 15.0),
                            (5, 128, (0.03, 0.5, 0.06), 15.0),
                            (6, 256, (0.03, 0.5, 0.01), 15.0)):
    _name = f"3d-{_n}x{_n}x{_n}-set{_k}"
    WORKLOADS[_name] = Workload(
        name=_name, nx=_n, ny=_n, nz=_n, coarse=(8, 8, 8), sigma=2.0, corr=_corr,
        cov="spherical", angle_deg=_ang, lnk_mean=-1.0, law=1, c_or_eta=1.0,
        steps=3, t_stars=(0.4, 1.0, 2.0), basis=4, restriction=0, n_post=5, nl_tol=1e-6,
        seeds=tuple(range(20)))


# The batched ensemble: independent realisations with sigma drawn uniformly
# in [1, 4] and grid sizes drawn from a ladder between 32^3 and 128x128x64,
# each solved for one implicit step with the 4M-cell workload's options
# (Dirichlet W/E, (B4), MSFE, 5 ILU(0) post steps, tolerance 1e-8, the
# FP32 preconditioner in FP64 refinement), coarse blocks of 8^3.
ENSEMBLE_SHAPES = ((32, 32, 32), (48, 48, 32), (64, 48, 32), (64, 64, 32), (64, 64, 64),
                   (96, 64, 48), (96, 96, 48), (128, 96, 64), (128, 128, 64))


def ensemble_members(n=64, seed=0, precision=1):
    """The n member workloads of the ensemble (seeded draw of shapes and
    sigmas; member k uses field seed 1000 + k)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx, ny, nz = ENSEMBLE_SHAPES[int(rng.integers(len(ENSEMBLE_SHAPES)))]
        sigma = float(rng.uniform(1.0, 4.0))
        out.append(Workload(
            name=f"ensemble-{k}-{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, coarse=(8, 8, 8),
            sigma=sigma, corr=(0.1, 0.1, 0.1), c_or_eta=0.1, steps=1, basis=4, restriction=0,
            n_post=5, nl_tol=1e-8, precision=precision, seeds=(1000 + k,)))
    return out


def line_columns(w: Workload):
    """Cells and values of the two prescribed columns of Test Case 2: the
    column (0, 0, z) at p_west and the column (nx-1, ny-1, z) at p_east."""
    z = np.arange(w.nz, dtype=np.int64)
    a = 0 + w.nx * (0 + w.ny * z)
    b = (w.nx - 1) + w.nx * ((w.ny - 1) + w.ny * z)
    cells = np.concatenate([a, b]).astype(np.int32)
    vals = np.concatenate([np.full(w.nz, w.p_west), np.full(w.nz, w.p_east)])
    return cells, vals


def _cell_transmissibility_sum(w: Workload, kx, ky, kz, h):
    """Sum over the internal faces of each cell of A_f / (h/(2k_a) + h/(2k_b))
    (cubic cells, mu = 1); only used to size the well rates."""
    shp = (w.nz, w.ny, w.nx)
    out = np.zeros(shp)
    for k, ax in ((kx, 2), (ky, 1), (kz, 0)):
        kk = np.asarray(k).reshape(shp)
        if kk.shape[ax] < 2:
            continue
        a = np.take(kk, np.arange(kk.shape[ax] - 1), axis=ax)
        b = np.take(kk, np.arange(1, kk.shape[ax]), axis=ax)
        t = (h * h) / (h / (2 * a) + h / (2 * b))
        lo = [slice(None)] * 3; lo[ax] = slice(0, kk.shape[ax] - 1)
        hi = [slice(None)] * 3; hi[ax] = slice(1, kk.shape[ax])
        out[tuple(lo)] += t
        out[tuple(hi)] += t
    return out.ravel()


def make_inputs(w: Workload, seed: int | None = None):
    """Concrete arrays and scalars for one realisation of workload w.

    Returns a dict with grid spacing, kx/ky/kz (float64, length N, index
    x + nx*(y + ny*z)), the first time step dt and every step's (dts), the
    initial pressure p0 (zero, as
    in Sec. 4.1.3), the source list (cell ids and volumetric rates q_i dV_i)
    and the prescribed cells with their pressures.
    """
    seed = w.seeds[0] if seed is None else seed
    kx, ky, kz = lognormal_permeability(
        w.nx, w.ny, w.nz, w.sigma, w.corr, seed, mean=w.lnk_mean, kind=w.cov,
        kz_ratio=w.kz_ratio, angle_deg=w.angle_deg)
    h = 1.0 / w.nx
    k_bar = math.exp(float(np.mean(np.log(kx))))
    dp = 1.0
    tau = w.mu * w.phi * w.alpha ** 2 / (k_bar * dp)
    if w.t_stars:
        ends = [0.0] + [float(t) for t in w.t_stars]
        dts = [(b - a) * tau for a, b in zip(ends[:-1], ends[1:])]
    else:
        dts = [w.dt_star * tau] * w.steps
    dt = dts[0]
    src_cell = np.zeros(0, dtype=np.int32)
    src_rate = np.zeros(0, dtype=np.float64)
    fix_cell = np.zeros(0, dtype=np.int32)
    fix_value = np.zeros(0, dtype=np.float64)
    if w.bc == "lines":
        fix_cell, fix_value = line_columns(w)
    if w.bc == "wells":
        # Vertical line wells through all layers at columns (0,0) (injector)
        # and (nx-1, ny-1) (producer).  Rates are fixed for the whole run.
        # Each perforated cell gets the rate that a pressure difference of
        # well_rate across all of its internal faces would drive,
        # q_i dV_i = +-well_rate * sum_faces T (TPFA, harmonic k average), so
        # that pressures stay O(well_rate) whatever the realisation.
        inj = np.array([0 + w.nx * (0 + w.ny * z) for z in range(w.nz)], np.int64)
        prod = np.array([(w.nx - 1) + w.nx * ((w.ny - 1) + w.ny * z) for z in range(w.nz)], np.int64)
        src_cell = np.concatenate([inj, prod]).astype(np.int32)
        tsum = _cell_transmissibility_sum(w, kx, ky, kz, h)
        src_rate = np.concatenate([w.well_rate * tsum[inj], -w.well_rate * tsum[prod]])
    return dict(
        nx=w.nx, ny=w.ny, nz=w.nz, dx=w.alpha * h, dy=h, dz=h,
        kx=kx, ky=ky, kz=kz, dt=dt, dts=dts, tau=tau, k_bar=k_bar,
        p0=np.zeros(w.n_cells), src_cell=src_cell, src_rate=src_rate,
        fix_cell=fix_cell, fix_value=fix_value,
        dirichlet=(w.bc == "dirichlet_we"), p_west=w.p_west, p_east=w.p_east,
    )
