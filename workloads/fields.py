"""Seeded Gaussian random fields for ln k (synthetic stand-ins for the paper's
sequential-Gaussian-simulation permeability sets, Sec. 4 and Table 2).

The paper draws ln k with spherical variograms (variance 4, mean -1) from
SGeMS; those realisations are not available, so fields are generated here by
circulant embedding of a stationary covariance on a periodic grid twice the
size of the domain in every active direction (Dietrich & Newsam's method).
Exponential and spherical covariances are both supported.  Negative
eigenvalues of the embedding (rare for these correlation lengths) are clipped
to zero, which makes the field an approximation of the target covariance.
"""
from __future__ import annotations

import numpy as np


def _covariance(h: np.ndarray, kind: str) -> np.ndarray:
    """Correlation function of the scaled lag h = |r / l| (unit variance)."""
    if kind == "exponential":
        return np.exp(-h)
    if kind == "spherical":
        return np.where(h < 1.0, 1.0 - 1.5 * h + 0.5 * h ** 3, 0.0)
    raise ValueError(f"unknown covariance {kind!r}")


def gaussian_field(shape_zyx, corr_cells_zyx, sigma, seed, mean=0.0,
                   kind="exponential", angle_deg=0.0):
    """Stationary Gaussian field on a (nz, ny, nx) grid.

    corr_cells_zyx: correlation lengths in cells along (z, y, x).
    angle_deg: rotation of the horizontal principal axes about z (layered
    sets of the paper use 15 degrees).
    Returns float64 array of shape (nz, ny, nx); C-order ravel gives the
    cell index i = x + nx*(y + ny*z).
    """
    shape = tuple(int(s) for s in shape_zyx)
    emb = tuple(2 * s if s > 1 else 1 for s in shape)
    # signed minimum-image lags on the periodic embedding grid
    lags = []
    for m in emb:
        a = np.arange(m, dtype=np.float64)
        lags.append(np.where(a <= m // 2, a, a - m))
    sz, sy, sx = np.meshgrid(*lags, indexing="ij")
    lz, ly, lx = (float(c) for c in corr_cells_zyx)
    th = np.deg2rad(angle_deg)
    u = np.cos(th) * sx + np.sin(th) * sy
    v = -np.sin(th) * sx + np.cos(th) * sy
    h = np.sqrt((u / lx) ** 2 + (v / ly) ** 2 + (sz / lz) ** 2)
    cov = sigma ** 2 * _covariance(h, kind)
    lam = np.fft.fftn(cov).real
    np.maximum(lam, 0.0, out=lam)
    m_tot = float(np.prod(emb))
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(emb) + 1j * rng.standard_normal(emb)
    y = np.fft.fftn(np.sqrt(lam / m_tot) * z).real
    return np.ascontiguousarray(y[: shape[0], : shape[1], : shape[2]] + mean)


def lognormal_permeability(nx, ny, nz, sigma, corr_frac_xyz, seed, mean=0.0,
                           kind="exponential", kz_ratio=1.0, angle_deg=0.0):
    """Return (kx, ky, kz) flattened float64 arrays of length nx*ny*nz.

    corr_frac_xyz: correlation lengths as fractions of the x-extent of the
    domain (the unit length), converted to cells with h = 1/nx.
    kz = kz_ratio * kx (vertical anisotropy); kx = ky.
    """
    corr_cells = (corr_frac_xyz[2] * nx, corr_frac_xyz[1] * nx, corr_frac_xyz[0] * nx)
    lnk = gaussian_field((nz, ny, nx), corr_cells, sigma, seed, mean=mean,
                         kind=kind, angle_deg=angle_deg)
    k = np.exp(lnk).ravel()
    return k, k.copy(), kz_ratio * k
