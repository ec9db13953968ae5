"""Z-slab decomposition of one (mesh, grid) problem over the ranks of a process group.

A grid point's value depends only on the features within w of it, so rank r can evaluate the
z-slab [k0, k1) of the grid with the features of the whole mesh and no exchange in the forward.
The vertex adjoint is a sum over band points, so the ranks' partial gradients are summed with one
all-reduce.  Every rank builds the features of the whole mesh (the build is small next to the
grid).  This module holds the host-side logic only: slab bounds, the slab's grid, the gradient
reduction, and the per-rank forward and backward through the library's C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Grid, sdf_narrow_band, sdf_narrow_band_backward


def slab_bounds(nz: int, world: int, rank: int) -> tuple[int, int]:
    """Balanced split of the nz grid layers: rank r gets [k0, k1), the first nz % world ranks one
    layer more; the slabs of all ranks tile [0, nz) without overlap."""
    if world < 1 or not 0 <= rank < world or nz < 0:
        raise ValueError("bad slab request")
    base, rem = divmod(nz, world)
    k0 = rank * base + min(rank, rem)
    return k0, k0 + base + (1 if rank < rem else 0)


def slab_grid(grid: Grid, world: int, rank: int) -> Grid:
    """The grid of rank r's slab: the same x-y layout and spacing, layers k0..k1-1, its origin moved
    up by k0 cells (float32, as the library stores it)."""
    k0, k1 = slab_bounds(grid.nz, world, rank)
    oz = float(np.float32(np.float32(grid.origin[2]) + np.float32(k0) * np.float32(grid.h)))
    return Grid(grid.nx, grid.ny, k1 - k0, (grid.origin[0], grid.origin[1], oz), grid.h)


def all_reduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum t over the ranks of the process group in place (no-op for a single process)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def forward(features, grid: Grid, w: float, world: int, rank: int, winner: bool = False, flags: int = 0):
    """This rank's slab of the narrow band: (slab grid, dist [, winner])."""
    g = slab_grid(grid, world, rank)
    return g, sdf_narrow_band(features, g, w, winner=winner, flags=flags)


def backward(features, grid: Grid, w: float, world: int, rank: int, grad_slab: torch.Tensor,
             winner_slab: torch.Tensor | None = None, group=None) -> torch.Tensor:
    """dL/d(welded vertices) of the whole grid: this rank's slab adjoint, summed over the ranks."""
    g = slab_grid(grid, world, rank)
    gv = sdf_narrow_band_backward(features, g, w, grad_slab, winner=winner_slab)
    return all_reduce_sum(gv, group)
