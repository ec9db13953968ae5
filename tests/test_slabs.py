"""Host logic of the z-slab decomposition (multi-GPU design, one slab per rank): slab bounds, slab
grids, and the gradient all-reduce, run as two gloo ranks on the CPU.  The FP64 oracle stands in
for each rank's GPU work: the ranks' slab bands must reassemble the whole grid's band, and the
all-reduced slab adjoints must equal the whole grid's adjoint."""
import os
import socket

import numpy as np
import pytest
import torch

import meshgen
from paper_1903_00353_gb300 import Grid, slabs


@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("nz", [1, 7, 64, 513])
def test_slab_bounds_tile_the_grid(nz, world):
    covered = []
    sizes = []
    for r in range(world):
        k0, k1 = slabs.slab_bounds(nz, world, r)
        assert 0 <= k0 <= k1 <= nz
        assert k0 % slabs.SLAB_ALIGN == 0 or k0 == nz  # slab starts on a tile layer
        covered.extend(range(k0, k1))
        sizes.append(k1 - k0)
    assert covered == list(range(nz))
    assert max(sizes) - min(sizes) < 2 * slabs.SLAB_ALIGN  # balanced to a block of layers (plus a partial last one)


def test_slab_grid_origin_and_shape():
    g = Grid(40, 30, 33, (0.25, 0.5, 0.125), 0.0137)
    total = 0
    for r in range(4):
        s = slabs.slab_grid(g, 4, r)
        k0, k1 = slabs.slab_bounds(33, 4, r)
        # the slab keeps the whole grid's origin and spacing and names its first layer
        assert (s.nx, s.ny, s.nz, s.h, s.k0) == (40, 30, k1 - k0, g.h, k0)
        assert s.origin == g.origin
        total += s.nz
    assert total == 33
    with pytest.raises(ValueError):
        slabs.slab_bounds(10, 2, 2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        soup = meshgen.config_soup(1)
        grid = Grid.cube(32)
        w = 3 / 32
        om = oracle.OracleMesh.from_soup(soup)
        sg = slabs.slab_grid(grid, world, rank)
        dims = (sg.nx, sg.ny, sg.nz)
        # the oracle's grid of the slab: the slab's points at the whole grid's positions
        org = (sg.origin[0], sg.origin[1], sg.origin[2] + sg.k0 * sg.h)
        d = om.narrow_band(dims, org, sg.h, w).ravel()
        pts = oracle.grid_points(dims, org, sg.h, np.arange(d.size))
        g = np.where(np.isfinite(d), 2.0 * (d - 0.01), 0.0)
        gv = torch.from_numpy(om.adjoint_points(pts, g, w))
        slabs.all_reduce_sum(gv)
        parts = [None] * world
        dist.all_gather_object(parts, d)
        if rank == 0:
            np.save(os.path.join(out_dir, "gv.npy"), gv.numpy())
            np.save(os.path.join(out_dir, "band.npy"), np.concatenate(parts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_band_and_adjoint(tmp_path):
    oracle = pytest.importorskip("oracle")
    world = 2
    torch.multiprocessing.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    soup = meshgen.config_soup(1)
    grid = Grid.cube(32)
    w = 3 / 32
    om = oracle.OracleMesh.from_soup(soup)
    dims = (grid.nx, grid.ny, grid.nz)
    d = om.narrow_band(dims, grid.origin, grid.h, w).ravel()
    band = np.load(tmp_path / "band.npy")
    # slabs are z ranges of an x-fastest layout: their concatenation is the whole grid
    assert band.shape == d.shape
    assert np.array_equal(np.isfinite(band), np.isfinite(d))
    assert np.array_equal(band[np.isfinite(d)], d[np.isfinite(d)])
    pts = oracle.grid_points(dims, grid.origin, grid.h, np.arange(d.size))
    g = np.where(np.isfinite(d), 2.0 * (d - 0.01), 0.0)
    gv_full = om.adjoint_points(pts, g, w)
    gv = np.load(tmp_path / "gv.npy")
    assert np.abs(gv).max() > 0
    np.testing.assert_allclose(gv, gv_full, rtol=1e-10, atol=1e-12 * np.abs(gv_full).max())
