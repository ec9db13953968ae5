"""Z-slab decomposition of one (mesh, grid) problem over the ranks of a process group.

A grid point's value depends only on the features within w of it, so rank r can evaluate the
z-slab [k0, k1) of the grid with the features of the whole mesh and no exchange in the forward.
The vertex adjoint is a sum over band points, so the ranks' partial gradients are summed with one
all-reduce.  Every rank builds the features of the whole mesh (the build is small next to the
grid).  This module holds the host-side logic only: slab bounds, the slab's grid, the gradient
reduction, and the per-rank forward and backward through the library's C ABI.
"""
from __future__ import annotations

import torch

from . import Grid, sdf_narrow_band, sdf_narrow_band_backward


# Slab boundaries fall on multiples of the tile kernel's tile depth along z, so that the slabs' tiles
# are the whole grid's tiles and the slabs reproduce it bit for bit.
SLAB_ALIGN = 8


def slab_bounds(nz: int, world: int, rank: int, align: int = SLAB_ALIGN) -> tuple[int, int]:
    """Balanced split of the nz grid layers in blocks of `align` layers: rank r gets [k0, k1), the
    first ranks one block more; the slabs of all ranks tile [0, nz) without overlap (a rank may get
    an empty slab when there are fewer blocks than ranks)."""
    if world < 1 or not 0 <= rank < world or nz < 0 or align < 1:
        raise ValueError("bad slab request")
    blocks = (nz + align - 1) // align
    base, rem = divmod(blocks, world)
    b0 = rank * base + min(rank, rem)
    b1 = b0 + base + (1 if rank < rem else 0)
    return min(nz, b0 * align), min(nz, b1 * align)


def slab_grid(grid: Grid, world: int, rank: int) -> Grid:
    """The grid of rank r's slab: the same origin, spacing and x-y layout, layers k0..k1-1 of the
    whole grid (sdf_grid's k0), so its points are exactly the whole grid's."""
    k0, k1 = slab_bounds(grid.nz, world, rank)
    return Grid(grid.nx, grid.ny, k1 - k0, grid.origin, grid.h, grid.k0 + k0)


def all_reduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum t over the ranks of the process group in place (no-op for a single process)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def forward(features, grid: Grid, w: float, world: int, rank: int, winner: bool = False, flags: int = 0):
    """This rank's slab of the narrow band: (slab grid, dist [, winner]); a rank whose slab is empty
    (fewer blocks of layers than ranks) gets empty tensors."""
    g = slab_grid(grid, world, rank)
    if g.nz == 0:
        empty = torch.empty((0, grid.ny, grid.nx), dtype=torch.float32, device="cuda")
        return g, ((empty, torch.empty(empty.shape, dtype=torch.int32, device="cuda")) if winner else empty)
    return g, sdf_narrow_band(features, g, w, winner=winner, flags=flags)


def backward(features, grid: Grid, w: float, world: int, rank: int, grad_slab: torch.Tensor,
             winner_slab: torch.Tensor | None = None, group=None) -> torch.Tensor:
    """dL/d(welded vertices) of the whole grid: this rank's slab adjoint, summed over the ranks."""
    g = slab_grid(grid, world, rank)
    if g.nz == 0:
        gv = torch.zeros(features.n_vert, 3, dtype=torch.float32, device="cuda")
    else:
        gv = sdf_narrow_band_backward(features, g, w, grad_slab, winner=winner_slab)
    return all_reduce_sum(gv, group)
