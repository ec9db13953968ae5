"""A loop that builds, evaluates and destroys a handle per step (a fitting or benchmark loop).

After its first steps such a loop takes no memory from the library's device pool: the destroyed
handle's scratch of its narrow-band calls, its array block and counters, and each build's own
scratch are kept for the next step (sdf_features_destroy in include/sdf.h).  The results of every
step are bitwise the same.  GPU only.
"""
import pytest
import torch

import meshgen
import paper_1903_00353_gb300 as sdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_build_per_step_loop_takes_no_pool_memory_after_warm_up():
    soup = torch.from_numpy(meshgen.torus(nu=120, nv=48, seed=11).soup(seed=12)).cuda()
    grid, w = sdf.Grid.cube(128), 3.0 / 128
    dist = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
    win = torch.empty(grid.shape, dtype=torch.int32, device="cuda")
    ref = None
    allocs = []
    for step in range(6):
        f = sdf.sdf_build_features(soup)
        sdf.sdf_narrow_band(f, grid, w, out=dist, winner=win)
        torch.cuda.synchronize()
        if ref is None:
            ref = (dist.clone(), win.clone(), f.vertex_map())
        else:
            assert torch.equal(dist, ref[0]) and torch.equal(win, ref[1])
            assert torch.equal(f.vertex_map(), ref[2])
        f.destroy()
        allocs.append(sdf.memory_stats()["pool_allocs"])
    # the first two steps may fill the kept blocks and plans; the last four take nothing new
    assert allocs[-1] == allocs[2], allocs
