"""Sign beyond the band (SDF_FLAG_FILL_SIGN): every point outside the band carries the
inside/outside sign of the FP64 oracle's full signed distance, the band itself is unchanged, and
batches agree with single calls.  GPU only."""
import numpy as np
import pytest
import torch

import meshgen
import oracle
import paper_1903_00353_gb300 as sdf
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def f32(x: float) -> float:
    return float(np.float32(x))


def grid_points(g):
    i = (np.arange(g.nx) + 0.5) * g.h + g.origin[0]
    j = (np.arange(g.ny) + 0.5) * g.h + g.origin[1]
    k = (np.arange(g.nz) + 0.5) * g.h + g.origin[2]
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    return np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)


CASES = {
    # grid covering the whole mesh
    "icosphere_64": (lambda: meshgen.config_mesh(1), lambda: sdf.Grid.cube(64), 3.0),
    # a torus: rows through the hole, rows inside the tube
    "torus_ragged": (lambda: meshgen.torus(nu=60, nv=24, seed=5),
                     lambda: sdf.Grid(90, 77, 45, (0.0, 0.0, f32(0.28)), f32(1 / 88)), 3.0),
    # several components
    "box_cluster": (lambda: meshgen.box_cluster(3, 2000, seed=7), lambda: sdf.Grid.cube(80), 2.5),
    "box_union": (lambda: meshgen.box_union(4, 2000, seed=6), lambda: sdf.Grid.cube(72), 3.0),
    # the grid lies partly deep inside a large sphere: whole rows and slabs without band points
    "inside_window": (lambda: meshgen.icosphere(12, radius=0.45),
                      lambda: sdf.Grid(40, 36, 33, (f32(0.3), f32(0.31), f32(0.05)), f32(1 / 100)), 3.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fill_sign_matches_oracle(name):
    mk, mg, cells = CASES[name]
    soup = mk().soup(seed=3)
    grid = mg()
    w = f32(cells * grid.h)
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    plain = sdf.sdf_narrow_band(feats, grid, w).cpu().numpy().ravel()
    filled = sdf.sdf_narrow_band(feats, grid, w, flags=sdf.FLAG_FILL_SIGN).cpu().numpy().ravel()
    band = np.isfinite(plain)
    # the band is untouched, bit for bit
    assert np.array_equal(plain[band].view(np.uint32), filled[band].view(np.uint32))
    assert np.all(np.isinf(filled[~band]))
    om = oracle.OracleMesh.from_soup(soup)
    d, _, _ = om.sdf_points(grid_points(grid))
    out = ~band
    assert np.all(np.abs(d[out]) >= w * (1 - 1e-5))  # points outside the band are far from the surface
    sign_gpu = np.where(filled[out] < 0, -1, 1)
    sign_or = np.where(d[out] < 0, -1, 1)
    bad = np.count_nonzero(sign_gpu != sign_or)
    assert bad == 0, f"{bad} of {out.sum()} points outside the band have the wrong sign"
    assert (filled[out] < 0).any() or name == "icosphere_64" or name == "box_cluster"
    # the band itself (identical in both calls) still matches the oracle
    parity.assert_parity(parity.compare(plain, np.where(np.abs(d) < w + 2 * grid.h, d, np.inf), w, grid.h))


def test_fill_sign_batch_equals_singles():
    meshes = [meshgen.config_mesh(1), meshgen.torus(nu=60, nv=24, seed=5), meshgen.box_cluster(2, 1500, seed=9)]
    grids = [sdf.Grid.cube(64), sdf.Grid(90, 77, 45, (0.0, 0.0, f32(0.28)), f32(1 / 88)), sdf.Grid.cube(48)]
    ws = [f32(3 * g.h) for g in grids]
    feats = [sdf.sdf_build_features(torch.from_numpy(m.soup(seed=4)).cuda()) for m in meshes]
    singles = [sdf.sdf_narrow_band(f, g, w, flags=sdf.FLAG_FILL_SIGN).clone() for f, g, w in zip(feats, grids, ws)]
    listed = sdf.sdf_narrow_band(feats, grids, ws, flags=sdf.FLAG_FILL_SIGN)
    batch = sdf.sdf_batch_create(feats, grids, ws, fill_sign=True)
    torch.cuda.synchronize()
    for a, b, c in zip(singles, listed, batch.outs):
        assert torch.equal(a, b) and torch.equal(a, c)
    for o in batch.outs:
        o.fill_(7.0)
    batch.run()
    torch.cuda.synchronize()
    for a, c in zip(singles, batch.outs):
        assert torch.equal(a, c)
    batch.destroy()


def test_fill_sign_needs_band_wider_than_step():
    feats = sdf.sdf_build_features(torch.from_numpy(meshgen.config_soup(1)).cuda())
    grid = sdf.Grid.cube(64)
    with pytest.raises(sdf.SDFError):
        sdf.sdf_narrow_band(feats, grid, f32(0.9 / 64), flags=sdf.FLAG_FILL_SIGN)
    sdf.sdf_narrow_band(feats, grid, f32(0.9 / 64))  # without the fill a narrow band is fine
