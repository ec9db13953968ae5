"""The z-slab decomposition on one GPU: the slabs' bands, evaluated one after another, reassemble
the whole grid's band, and their adjoints sum to the whole grid's adjoint.  Slabs that start on a
tile boundary reproduce the whole grid bit for bit (dyadic spacing keeps the slab origins exact);
other slabs tile the grid differently, so inclusion decisions inside the tolerance margin may
pick another of two near-equal candidates: they agree within the parity tolerance.  GPU only."""
import numpy as np
import pytest
import torch

import meshgen
import paper_1903_00353_gb300 as sdf
from paper_1903_00353_gb300 import slabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_reassemble_forward_and_adjoint(world):
    soup = meshgen.config_soup(2)
    grid = sdf.Grid.cube(128)
    w = 4 / 128
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    full, win = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    g_full = torch.where(torch.isfinite(full), 2.0 * (full - 0.01), torch.zeros_like(full))
    gv_full = sdf.sdf_narrow_band_backward(feats, grid, w, g_full, winner=win)
    parts, gv = [], torch.zeros_like(gv_full)
    for r in range(world):
        sg, (d, wn) = slabs.forward(feats, grid, w, world, r, winner=True)
        parts.append(d)
        gs = torch.where(torch.isfinite(d), 2.0 * (d - 0.01), torch.zeros_like(d))
        gv += sdf.sdf_narrow_band_backward(feats, sg, w, gs, winner=wn)
    joined = torch.cat(parts, dim=0)
    if all(slabs.slab_bounds(grid.nz, world, r)[0] % 8 == 0 for r in range(world)):
        assert torch.equal(joined, full)
    a, b = joined.cpu().numpy().ravel(), full.cpu().numpy().ravel()
    fa, fb = np.isfinite(a), np.isfinite(b)
    edge = np.abs(np.abs(np.where(fb, b, a)) - w) <= 1e-5 * grid.h
    assert np.all((fa == fb) | edge)
    both = fa & fb
    assert np.abs(a[both] - b[both]).max() <= 2e-6
    rel = float((gv - gv_full).norm() / gv_full.norm())
    assert rel < 1e-5, rel
