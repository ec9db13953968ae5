"""Compact band list (sdf_narrow_band_list): the list holds every band point of the dense field
exactly once with its winner (including the points the FP64 re-decision moves into the band), an
overflow is reported and grown, and the adjoint and the fused L2 loss over the list equal the
dense path's and the FP64 oracle's.  GPU only."""
import ctypes

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


CASES = {
    # vector rows (nx a multiple of 4)
    "icosphere_c1": (lambda: meshgen.config_mesh(1), lambda: sdf.Grid.cube(64), 3.0),
    # scalar rows (nx = 90), non-dyadic spacing
    "torus_ragged": (lambda: meshgen.torus(nu=60, nv=24, seed=5),
                     lambda: sdf.Grid(90, 77, 45, (0.0, 0.0, f32(0.28)), f32(1 / 88)), 3.0),
    "box_union": (lambda: meshgen.box_union(4, 2000, seed=6), lambda: sdf.Grid.cube(72), 3.0),
    "knot": (lambda: meshgen.knot_tube(n_along=600, n_around=16, seed=8), lambda: sdf.Grid.cube(96), 2.5),
}


def _case(name):
    mk, mg, cells = CASES[name]
    soup = mk().soup(seed=3)
    grid = mg()
    w = f32(cells * grid.h)
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    return soup, feats, grid, w


@pytest.mark.parametrize("name", sorted(CASES))
def test_list_holds_each_band_point_once_with_its_winner(name):
    soup, feats, grid, w = _case(name)
    d_ref, w_ref = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    d, bl, wn = sdf.sdf_narrow_band_list(feats, grid, w, winner=True)
    assert torch.equal(d, d_ref) and torch.equal(wn, w_ref)
    band = torch.nonzero(torch.isfinite(d_ref.view(-1))).view(-1)
    assert len(bl) == band.numel() > 0
    idx = bl.indices().long()
    order = torch.argsort(idx)
    assert torch.equal(idx[order], band)  # every band point, each once
    assert torch.equal(bl.winners().long(), w_ref.view(-1)[idx].long())
    # without dense winners: the same field and the same set of entries
    d2, bl2 = sdf.sdf_narrow_band_list(feats, grid, w)
    assert torch.equal(d2, d_ref)
    e1 = bl.entries[: len(bl)].long()
    e2 = bl2.entries[: len(bl2)].long()
    k1 = e1[:, 0] * (1 << 31) + e1[:, 1]
    k2 = e2[:, 0] * (1 << 31) + e2[:, 1]
    assert torch.equal(torch.sort(k1).values, torch.sort(k2).values)


def test_list_includes_points_decided_in_fp64():
    """A box whose faces pass through grid planes: the points on the faces (d = 0, inside the sign
    window) and those at exactly w from them (the band-edge window) are decided in FP64, and those
    that land in the band enter the list through the re-decision, not the tile kernel."""
    mesh = meshgen.box(center=(0.5, 0.5, 0.5), half=(12.5 / 64,) * 3, subdiv=2)
    feats = sdf.sdf_build_features(torch.from_numpy(mesh.soup(seed=1)).cuda())
    grid, w = sdf.Grid.cube(64), 3 / 64
    d_ref, w_ref = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    st = feats.status()
    assert st["fp64_points"] > 1000
    d, bl = sdf.sdf_narrow_band_list(feats, grid, w)
    assert torch.equal(d, d_ref)
    band = torch.nonzero(torch.isfinite(d_ref.view(-1))).view(-1)
    idx = bl.indices().long()
    assert torch.equal(torch.sort(idx).values, band)
    assert torch.equal(bl.winners().long(), w_ref.view(-1)[idx].long())
    assert bool((d_ref.view(-1)[band] == 0).any())  # face points, decided into the band


def test_list_overflow_is_reported_and_grown():
    soup, feats, grid, w = _case("torus_ragged")
    d_ref, w_ref = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    n_band = int(torch.isfinite(d_ref).sum())
    # through the C ABI with a short list and no synchronisation: nothing written past the
    # capacity, the count holds the band's length, the status reports the overflow
    bl = sdf.BandList(1000)
    bl.entries.fill_(-5)
    cap = 100
    ga = (sdf._CGrid * 1)(grid.c())
    dist = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
    code = sdf.load_library().sdf_narrow_band_list(
        feats.handle, ga, float(w), dist.data_ptr(), None, bl.entries.data_ptr(), cap, bl.count.data_ptr(),
        sdf.FLAG_NO_SYNC, sdf._stream())
    assert code == 0
    torch.cuda.synchronize()
    assert int(bl.count.item()) == n_band > cap
    assert bool((bl.entries[cap:] == -5).all())
    with pytest.raises(sdf.SDFError) as e:
        feats.status()
    assert e.value.code == sdf.ERR_LIST_OVERFLOW
    # synchronous: the call reports the overflow
    code = sdf.load_library().sdf_narrow_band_list(
        feats.handle, ga, float(w), dist.data_ptr(), None, bl.entries.data_ptr(), cap, bl.count.data_ptr(), 0,
        sdf._stream())
    assert code == sdf.ERR_LIST_OVERFLOW
    # the binding grows the list and repeats the call
    d, bl2 = sdf.sdf_narrow_band_list(feats, grid, w, band_list=sdf.BandList(10))
    assert torch.equal(d, d_ref) and len(bl2) == n_band and bl2.capacity >= n_band
    feats.status()  # the repeated call left no overflow behind


def test_list_rejects_the_cell_loop_and_large_grids():
    soup, feats, grid, w = _case("icosphere_c1")
    with pytest.raises(sdf.SDFError):
        sdf.sdf_narrow_band_list(feats, grid, w, flags=sdf.FLAG_CELL_LOOP)
    big = sdf.Grid(2048, 2048, 1025, (0.0, 0.0, 0.0), 1 / 2048)  # more than 2^32 points
    ga = (sdf._CGrid * 1)(big.c())
    bl = sdf.BandList(16)
    code = sdf.load_library().sdf_narrow_band_list(feats.handle, ga, float(3 / 2048), ctypes.c_void_p(256), None,
                                                   bl.entries.data_ptr(), 16, bl.count.data_ptr(), 0, sdf._stream())
    assert code == 5  # SDF_ERR_TOO_LARGE, before any device work


@pytest.mark.parametrize("name", ["icosphere_c1", "torus_ragged", "box_union"])
def test_list_adjoint_and_fused_l2_equal_the_dense_path(name):
    soup, feats, grid, w = _case(name)
    d, bl, wn = sdf.sdf_narrow_band_list(feats, grid, w, winner=True)
    gen = torch.Generator(device="cuda").manual_seed(5)
    target = (torch.rand(grid.shape, device="cuda", generator=gen) - 0.5) * 0.02
    loss_d, g, band_d = sdf.band_l2_loss(d, target)
    gv_dense = sdf.sdf_narrow_band_backward(feats, grid, w, g, winner=wn)
    gv_list = sdf.band_list_backward(feats, grid, bl, g)
    scale = float(gv_dense.norm())
    assert scale > 0
    assert float((gv_list - gv_dense).norm()) <= 1e-5 * scale
    loss_l, gv_fused, band_l = sdf.band_list_l2(feats, grid, bl, d, target)
    assert int(band_l) == int(band_d) == len(bl)
    assert abs(float(loss_l) - float(loss_d)) <= 1e-12 * abs(float(loss_d))
    assert float((gv_fused - gv_dense).norm()) <= 1e-5 * scale
    # against the FP64 oracle's adjoint of the same loss at the same band points
    idx = bl.indices().long()
    gp = (2.0 * (d.view(-1)[idx] - target.view(-1)[idx])).double().cpu().numpy()
    pts = oracle.grid_points((grid.nx, grid.ny, grid.nz), grid.origin, grid.h, idx.cpu().numpy())
    om = oracle.OracleMesh.from_soup(soup)
    go = om.adjoint_points(pts, gp, w + 1e-9)
    a = gv_fused.cpu().numpy()[feats.vertex_map().cpu().numpy()]
    b = go[om.soup_vid()]
    assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)


def test_fused_list_fit_step_matches_the_dense_fit_step():
    """One shape-fitting step with the list path (forward with list, fused loss and adjoint) equals
    the step with dense winners, the dense fused loss and the dense adjoint."""
    mesh = meshgen.icosphere(12, radius=0.3, displacement=0.02, seed=5)
    feats = sdf.sdf_build_features(torch.from_numpy(mesh.soup(seed=7)).cuda())
    grid, w = sdf.Grid.cube(128), 4 / 128
    c = (torch.arange(128, device="cuda", dtype=torch.float64) + 0.5) * grid.h
    Z, Y, X = torch.meshgrid(c, c, c, indexing="ij")
    target = meshgen.ellipsoid_sdf_torch(torch.stack([X, Y, Z], dim=-1)).to(torch.float32)
    d, wn = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    loss_d, g, _ = sdf.band_l2_loss(d, target)
    gv_d = sdf.sdf_narrow_band_backward(feats, grid, w, g, winner=wn)
    d2, bl = sdf.sdf_narrow_band_list(feats, grid, w, band_list=sdf.BandList(128 ** 3 // 4), flags=sdf.FLAG_NO_SYNC)
    loss_l, gv_l, _ = sdf.band_list_l2(feats, grid, bl, d2, target)
    feats.status()
    assert torch.equal(d, d2)
    assert abs(float(loss_l) - float(loss_d)) <= 1e-12 * float(loss_d)
    assert float((gv_l - gv_d).norm()) <= 1e-5 * float(gv_d.norm())


def test_fp64_gradient_accumulation():
    """SDF_FLAG_GRAD_F64 (a float64 grad_vertices): the same per-point contributions summed in FP64,
    so two runs agree to FP64 rounding whatever the order of the atomics, and the result is the
    FP32 accumulation's up to FP32 rounding; the dense adjoint and both list adjoints agree."""
    soup, feats, grid, w = _case("torus_ragged")
    d, bl, wn = sdf.sdf_narrow_band_list(feats, grid, w, winner=True)
    gen = torch.Generator(device="cuda").manual_seed(9)
    target = (torch.rand(grid.shape, device="cuda", generator=gen) - 0.5) * 0.02
    _, g, _ = sdf.band_l2_loss(d, target)
    gv32 = sdf.band_list_backward(feats, grid, bl, g)
    runs = []
    for _ in range(2):
        gv64 = torch.zeros(feats.n_vert, 3, dtype=torch.float64, device="cuda")
        runs.append(sdf.band_list_backward(feats, grid, bl, g, grad_vertices=gv64))
    scale = float(runs[0].norm())
    assert float((runs[0] - runs[1]).norm()) <= 1e-12 * scale
    assert float((runs[0] - gv32.double()).norm()) <= 1e-5 * scale
    dense64 = sdf.sdf_narrow_band_backward(feats, grid, w, g, winner=wn,
                                           grad_vertices=torch.zeros_like(runs[0]))
    assert float((dense64 - runs[0]).norm()) <= 1e-12 * scale
    _, fused64, _ = sdf.band_list_l2(feats, grid, bl, d, target, grad_vertices=torch.zeros_like(runs[0]))
    assert float((fused64 - runs[0]).norm()) <= 1e-6 * scale  # g formed in the kernel vs read (FP32)
    with pytest.raises(ValueError):
        sdf.band_list_backward(feats, grid, bl, g, grad_vertices=torch.zeros(3, 3, dtype=torch.float64,
                                                                             device="cuda"))


def test_batched_lists_equal_the_single_problem_fields_and_bands():
    """sdf_narrow_band_lists: a batch of three problems in one launch sequence, every list starting
    too short (grown by the binding after the call reports the overflow)."""
    names = ["icosphere_c1", "torus_ragged", "box_union"]
    cases = [_case(nm) for nm in names]
    feats, grids, ws = [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases]
    dists, lists = sdf.sdf_narrow_band_lists(feats, grids, ws, band_lists=[sdf.BandList(100) for _ in names])
    for f, g, w, d, bl in zip(feats, grids, ws, dists, lists):
        d_ref, w_ref = sdf.sdf_narrow_band(f, g, w, winner=True)
        assert torch.equal(d, d_ref)
        band = torch.nonzero(torch.isfinite(d_ref.view(-1))).view(-1)
        idx = bl.indices().long()
        assert len(bl) == band.numel() > 100
        assert torch.equal(torch.sort(idx).values, band)
        assert torch.equal(bl.winners().long(), w_ref.view(-1)[idx].long())


@pytest.mark.parametrize("case", ["c1_64", "torus_ragged", "c2_512", "c4_1024"])
def test_sparse_forward_matches_dense_and_oracle(case):
    """The sparse forward (band list with distances, no dense field): the same band points, winners
    and values as the dense forward, and the oracle's values at sampled list points."""
    if case == "c1_64":
        soup, grid, w = meshgen.config_soup(1), sdf.Grid.cube(64), 3 / 64
    elif case == "torus_ragged":
        soup = meshgen.torus(nu=60, nv=24, seed=3).soup(seed=2)
        h = float(np.float32(0.0123))
        grid, w = sdf.Grid(90, 77, 45, (0.0, 0.0, float(np.float32(0.23))), h), float(np.float32(3 * h))
    else:
        idx = 2 if case == "c2_512" else 4
        N, cells = meshgen.CONFIG_GRID[idx]
        soup, grid, w = meshgen.config_soup(idx), sdf.Grid.cube(N), cells / N
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    bl = sdf.sdf_narrow_band_sparse(feats, grid, w)
    n = len(bl)
    idx_s = bl.indices().long()
    order = torch.argsort(idx_s)
    idx_s, win_s, d_s = idx_s[order], bl.winners()[order], bl.dist[:n][order]
    dense, win = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    band = torch.nonzero(torch.isfinite(dense.view(-1))).view(-1)
    assert n == band.numel()
    assert torch.equal(idx_s, band)
    assert torch.equal(d_s, dense.view(-1)[band])
    assert torch.equal(win_s, win.view(-1)[band])
    del dense, win
    torch.cuda.empty_cache()
    # oracle at up to 20000 listed points
    rng = np.random.default_rng(5)
    pick = rng.choice(n, size=min(n, 20000), replace=False)
    ii = idx_s.cpu().numpy()[pick]
    om = oracle.OracleMesh.from_soup(soup)
    d_or, _, _ = om.band_points((grid.nx, grid.ny, grid.nz), grid.origin, grid.h, w + 2 * grid.h, ii)
    parity.assert_parity(parity.compare(d_s.cpu().numpy()[pick], d_or, w, grid.h))
