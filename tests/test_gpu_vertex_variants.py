"""The paper's vertex extrusions (cone around N_alpha, Sections 3.3 and 8.3; hemispheres, Section
4.3) in the cell-loop schedule, compared with the FP64 oracle.  What must hold for any extrusion
shape: every stored value is a true distance to a surface point, so no point outside the oracle's
band is stored and no stored |d| is below the true distance.  On a smooth convex mesh both shapes
cover the band completely.  The coverage on saddle and ruff vertices (where the paper leaves
correctness open) is measured and printed.  GPU only."""
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


MESHES = {
    "icosphere_c1": lambda: meshgen.config_mesh(1),
    "saddle": lambda: meshgen.star_fan_solid(8, [0.06, -0.06] * 4, apex_h=0.0),
    "ruff": lambda: meshgen.star_fan_solid(6, [0.25, -0.12] * 3, apex_h=0.05, bottom=-0.25),
    "torus": lambda: meshgen.torus(nu=40, nv=16, seed=7),
    "knot": lambda: meshgen.knot_tube(n_along=400, n_around=16, seed=8),
    "box_cluster": lambda: meshgen.box_cluster(2, 1500, seed=9),
    "box_union": lambda: meshgen.box_union(4, 2000, seed=6),
}
VARIANTS = {"cone": sdf.FLAG_VERTEX_CONE, "hemisphere": sdf.FLAG_VERTEX_HEMISPHERE}


def coverage(name, variant, N=64):
    soup = MESHES[name]().soup(seed=3)
    grid, w = sdf.Grid.cube(N), 3 / N
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    d = sdf.sdf_narrow_band(feats, grid, w, flags=sdf.FLAG_CELL_LOOP | VARIANTS[variant]).cpu().numpy().ravel()
    om = oracle.OracleMesh.from_soup(soup)
    ref = om.narrow_band((N, N, N), grid.origin, grid.h, w + 2 * grid.h).ravel()
    return d, ref, parity.compare(d, ref, w, grid.h), w, grid.h


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("name", sorted(MESHES))
def test_paper_vertex_extrusions_store_true_distances(name, variant):
    d, ref, st, w, h = coverage(name, variant)
    print(f"{name:14s} {variant:10s} band {st['band_oracle']:7d} missing {st['missing']:5d} "
          f"sign {st['sign_mismatch']:4d} max_err {st['max_abs_err']:.2e}")
    assert st["extra"] == 0
    both = np.isfinite(d) & np.isfinite(ref)
    assert np.all(np.abs(d[both]) >= np.abs(ref[both]) - 2e-6)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_paper_vertex_extrusions_cover_a_smooth_convex_mesh(variant):
    _, _, st, _, _ = coverage("icosphere_c1", variant)
    parity.assert_parity(st)


def test_variants_need_the_cell_loop():
    feats = sdf.sdf_build_features(torch.from_numpy(meshgen.config_soup(1)).cuda())
    with pytest.raises(sdf.SDFError):
        sdf.sdf_narrow_band(feats, sdf.Grid.cube(32), 3 / 32, flags=sdf.FLAG_VERTEX_CONE)
    with pytest.raises(sdf.SDFError):
        sdf.sdf_narrow_band(feats, sdf.Grid.cube(32), 3 / 32,
                            flags=sdf.FLAG_CELL_LOOP | sdf.FLAG_VERTEX_CONE | sdf.FLAG_VERTEX_HEMISPHERE)
