"""Primal- and dual-coarse grids of Sec. 3 (Fig. 1) and the wirebasket
classification used by the reduced-problem basis construction.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading R8 (the paper shows the grids only in a figure that is not
available): primal-coarse blocks are boxes of b_d fine cells along each
active direction d (b_d must divide n_d); the coarse node ("vertex") of
primal block I is the fine cell at offset floor(b_d/2) inside it, so vertex
coordinates along d are v_d(I) = I*b_d + floor(b_d/2).  Dual-coarse blocks
are the boxes spanned by neighbouring vertices; the slabs between the domain
boundary and the first/last vertex plane are partial dual blocks.

A fine cell's level is the number of active directions in which its
coordinate is NOT a vertex coordinate: 0 = vertex, 1 = edge, 2 = face,
3 = interior (in 2D the highest level is 2, in 1D it is 1).  Cells of one
level that share, in every direction, either the same vertex coordinate or
the same open interval between vertex coordinates form one local entity
(an edge segment, a face patch, or a dual-block interior).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .problem import Grid


@dataclass
class Entity:
    level: int
    cells: np.ndarray      # fine cell ids, ascending
    corners: np.ndarray    # coarse ids of the vertices spanning it, ascending


@dataclass
class Wirebasket:
    grid: Grid
    coarse: tuple          # (bx, by, bz)
    nc: tuple              # coarse cells per direction
    level: np.ndarray      # per fine cell
    entity: np.ndarray     # per fine cell: index into entities (-1 for vertices)
    entities: list
    vertex_cell: np.ndarray  # fine cell of coarse node J
    d_active: int

    @property
    def Nc(self) -> int:
        return int(np.prod(self.nc))

    def coarse_index(self, Jx, Jy, Jz):
        return Jx + self.nc[0] * (Jy + self.nc[1] * Jz)


def _check(n, b):
    if n == 1:
        if b != 1:
            raise ValueError("an inactive direction needs coarse size 1")
    elif b < 2 or n % b != 0:
        raise ValueError(f"coarse size {b} must be >= 2 and divide {n}")


def build_wirebasket(g: Grid, coarse) -> Wirebasket:
    n = (g.nx, g.ny, g.nz)
    b = tuple(int(v) for v in coarse)
    for nd, bd in zip(n, b):
        _check(nd, bd)
    nc = tuple(nd // bd for nd, bd in zip(n, b))
    off = tuple(bd // 2 for bd in b)
    coords = g.coords()
    active = [nd > 1 for nd in n]
    # per direction: on-lattice flag, vertex index (if on lattice) and the
    # interval index j (vertex planes j-1 and j bound it; 0 and nc are the
    # boundary slabs)
    on, key = [], []
    for d in range(3):
        x = coords[d]
        if not active[d]:
            on.append(np.ones(g.N, bool)); key.append(np.zeros(g.N, np.int64)); continue
        s = x - off[d]
        on_d = (s >= 0) & (s % b[d] == 0)
        j = np.where(s >= 0, s // b[d] + 1, 0)          # interval index for off-lattice x
        I = np.where(on_d, s // b[d], -1)               # vertex index for on-lattice x
        on.append(on_d)
        # encode "vertex I" as 2*I and "interval j" as 2*j - 1 so both fit one key
        key.append(np.where(on_d, 2 * I, 2 * j - 1))
    level = np.zeros(g.N, np.int64)
    for d in range(3):
        if active[d]:
            level += (~on[d]).astype(np.int64)
    # group cells into entities by (level, key_x, key_y, key_z)
    k3 = np.stack([level, key[0], key[1], key[2]], axis=1)
    uniq, inv = np.unique(k3, axis=0, return_inverse=True)
    inv = inv.ravel()
    order = np.argsort(inv, kind="stable")
    bounds = np.searchsorted(inv[order], np.arange(len(uniq) + 1))
    entity = np.full(g.N, -1, np.int64)
    entities = []
    for u in range(len(uniq)):
        lev = int(uniq[u, 0])
        if lev == 0:
            continue
        cells = np.sort(order[bounds[u]:bounds[u + 1]])
        # corner vertex indices per direction
        per_dir = []
        for d in range(3):
            kd = int(uniq[u, 1 + d])
            if not active[d]:
                per_dir.append([0])
            elif kd % 2 == 0:
                per_dir.append([kd // 2])
            else:
                j = (kd + 1) // 2
                per_dir.append([J for J in (j - 1, j) if 0 <= J < nc[d]])
        corners = sorted(Jx + nc[0] * (Jy + nc[1] * Jz)
                         for Jx in per_dir[0] for Jy in per_dir[1] for Jz in per_dir[2])
        entity[cells] = len(entities)
        entities.append(Entity(lev, cells, np.asarray(corners, np.int64)))
    # vertex cells and their coarse ids
    x, y, z = coords
    vcell = np.zeros(int(np.prod(nc)), np.int64)
    for Jz in range(nc[2]):
        for Jy in range(nc[1]):
            for Jx in range(nc[0]):
                vx = Jx * b[0] + off[0] if active[0] else 0
                vy = Jy * b[1] + off[1] if active[1] else 0
                vz = Jz * b[2] + off[2] if active[2] else 0
                vcell[Jx + nc[0] * (Jy + nc[1] * Jz)] = vx + g.nx * (vy + g.ny * vz)
    return Wirebasket(g, b, nc, level, entity, entities, vcell, int(sum(active)))
