"""Analytic TSDF volumes used as shared inputs (not produced by fusion).

A grid of nx x ny x nz nodes at origin + voxel_size * (i, j, k), stored
x-fastest (flat index i + nx * (j + ny * k)).  The value at a node is the
closed-form scene distance divided by the truncation and clamped to [-1, 1];
nodes deeper than one truncation inside matter are unobserved (weight 0).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rng import uniform01


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    voxel_size: float
    trunc: float
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def node_positions(self, k0: int = 0, k1: int | None = None) -> np.ndarray:
        """World positions of the nodes in z-slices k0..k1-1, shape (nz', ny, nx, 3)."""
        k1 = self.nz if k1 is None else k1
        i = np.arange(self.nx, dtype=np.float64)
        j = np.arange(self.ny, dtype=np.float64)
        k = np.arange(k0, k1, dtype=np.float64)
        kk, jj, ii = np.meshgrid(k, j, i, indexing="ij")
        o = np.asarray(self.origin, dtype=np.float64)
        return np.stack([o[0] + self.voxel_size * ii, o[1] + self.voxel_size * jj,
                         o[2] + self.voxel_size * kk], axis=-1)


def analytic_tsdf(scene, grid: Grid, hole_bricks: float = 0.0, seed: int = 0,
                  slab: int = 32):
    """(tsdf, weight) float32 arrays of length grid.n_nodes.

    `hole_bricks` marks that fraction of 8^3 bricks unobserved (seeded), to
    exercise the all-eight-nodes-observed rule."""
    tsdf = np.empty(grid.n_nodes, dtype=np.float32)
    weight = np.empty(grid.n_nodes, dtype=np.float32)
    plane = grid.nx * grid.ny
    for k0 in range(0, grid.nz, slab):
        k1 = min(grid.nz, k0 + slab)
        d = scene.sdf(grid.node_positions(k0, k1)).reshape(-1)
        t = np.clip(d / grid.trunc, -1.0, 1.0)
        w = (d > -grid.trunc).astype(np.float32)
        t = np.where(w > 0, t, 1.0)
        tsdf[k0 * plane:k1 * plane] = t
        weight[k0 * plane:k1 * plane] = w
    if hole_bricks > 0.0:
        bx, by, bz = (grid.nx + 7) // 8, (grid.ny + 7) // 8, (grid.nz + 7) // 8
        u = uniform01(7000 + seed, bx * by * bz).reshape(bz, by, bx)
        W = weight.reshape(grid.nz, grid.ny, grid.nx)
        T = tsdf.reshape(grid.nz, grid.ny, grid.nx)
        for kb, jb, ib in zip(*np.nonzero(u < hole_bricks)):
            sl = (slice(8 * kb, 8 * kb + 8), slice(8 * jb, 8 * jb + 8), slice(8 * ib, 8 * ib + 8))
            W[sl] = 0.0
            T[sl] = 1.0
    return tsdf, weight
