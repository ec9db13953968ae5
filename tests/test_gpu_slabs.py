"""The z-slab decomposition on one GPU: the slabs' bands, evaluated one after another, reassemble
the whole grid's band bit for bit (a slab keeps the whole grid's origin and names its first layer,
k0, and its layers start on tile boundaries, so its tiles and arithmetic are the whole grid's, on
any spacing), the reassembled field matches the FP64 oracle, and the slabs' adjoints sum to the
whole grid's adjoint.  GPU only."""
import numpy as np
import pytest
import torch

import meshgen
import oracle
import paper_1903_00353_gb300 as sdf
from paper_1903_00353_gb300 import slabs
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("world,spacing", [(2, "dyadic"), (3, "dyadic"), (3, "ragged"), (5, "ragged")])
def test_slabs_reassemble_forward_and_adjoint(world, spacing):
    soup = meshgen.config_soup(2)
    if spacing == "dyadic":
        grid, w = sdf.Grid.cube(128), 4 / 128
    else:
        h = float(np.float32(0.00813))
        grid = sdf.Grid(130, 121, 117, (float(np.float32(-0.021)), float(np.float32(0.013)), float(np.float32(0.0317))), h)
        w = float(np.float32(4 * h))
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
    assert torch.equal(joined, full)
    # the reassembled field against the oracle on the whole grid's points near the surface
    idx = parity.near_surface_indices(soup, (grid.nx, grid.ny, grid.nz), grid.origin, grid.h, w, 40_000, 353_777,
                                      n_uniform=4_000)
    om = oracle.OracleMesh.from_soup(soup)
    d_or, _, _ = om.band_points((grid.nx, grid.ny, grid.nz), grid.origin, grid.h, w + 2 * grid.h, idx)
    parity.assert_parity(parity.compare(joined.view(-1)[torch.from_numpy(idx).cuda()].cpu().numpy(), d_or, w, grid.h))
    rel = float((gv - gv_full).norm() / gv_full.norm())
    assert rel < 1e-5, rel
