"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.  GPU only."""
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


def gpu_band(soup_np, grid, w, flags=0, winner=False):
    feats = sdf.sdf_build_features(torch.from_numpy(soup_np).cuda(), flags=flags)
    res = sdf.sdf_narrow_band(feats, grid, w, winner=winner)
    torch.cuda.synchronize()
    return feats, res


def oracle_dense(soup_np, grid, w, ext_cells=2):
    om = oracle.OracleMesh.from_soup(soup_np)
    d = om.narrow_band((grid.nx, grid.ny, grid.nz), grid.origin, grid.h, w + ext_cells * grid.h)
    return om, d


def full_grid_case(soup_np, grid, w):
    feats, (dist, win) = gpu_band(soup_np, grid, w, winner=True)
    om, ref = oracle_dense(soup_np, grid, w)
    st = parity.compare(dist.cpu().numpy(), ref, w, grid.h)
    parity.assert_parity(st)
    assert st["band_oracle"] > 0
    w_np = win.cpu().numpy().ravel()
    band = np.isfinite(dist.cpu().numpy().ravel())
    n_feat = feats.n_tri + feats.n_edge + feats.n_vert
    assert np.all(w_np[~band] == -1)
    assert np.all((w_np[band] >= 0) & (w_np[band] < n_feat))
    return feats, om, st


TINY = {
    "tetra": lambda: meshgen.regular_tetrahedron(size=0.2),
    "cube_flat": lambda: meshgen.box(half=(0.2, 0.15, 0.1), subdiv=3),
    "octa": lambda: meshgen.octahedron(size=0.25),
    "saddle": lambda: meshgen.star_fan_solid(8, [0.06, -0.06] * 4, apex_h=0.0),
    "ruff": lambda: meshgen.star_fan_solid(6, [0.25, -0.12] * 3, apex_h=0.05, bottom=-0.25),
    "torus_small": lambda: meshgen.torus(nu=40, nv=16, seed=7),
    "knot_small": lambda: meshgen.knot_tube(n_along=400, n_around=16, seed=8),
    # overlapping rotated boxes: concave creases, saddle vertices where a crease meets a box edge
    "box_union3": lambda: meshgen.box_union(3, 1500, seed=2),
    "box_union4": lambda: meshgen.box_union(4, 3000, seed=3),
    # a dense cluster (36k vertices within a few micro-units) next to large triangles: long runs of
    # distinct vertices under one weld key, sorted by the block-wide fix-up
    "dense_cluster": lambda: meshgen.dense_cluster(),
}


def test_c1_icosphere_full_grid():
    soup = meshgen.config_soup(1)
    feats, om, st = full_grid_case(soup, sdf.Grid.cube(64), 3 / 64)
    assert feats.n_vert == om.V == 162 and feats.n_edge == om.E == 480
    print(st)


@pytest.mark.parametrize("name", sorted(TINY))
def test_small_meshes_full_grid_dyadic(name):
    soup = TINY[name]().soup(seed=3)
    full_grid_case(soup, sdf.Grid.cube(64), 3 / 64)


@pytest.mark.parametrize("name", ["torus_small", "saddle", "cube_flat", "knot_small", "box_union4"])
def test_ragged_grid_nondyadic_spacing(name):
    soup = TINY[name]().soup(seed=4)
    h = f32(0.0137)
    grid = sdf.Grid(70, 45, 75, (f32(-0.013), f32(0.021), f32(0.0071)), h)
    full_grid_case(soup, grid, f32(2.5 * h))


def test_classification_and_weld_match_oracle():
    for mesh in (meshgen.torus(nu=60, nv=24, seed=2), meshgen.knot_tube(n_along=600, n_around=20, seed=5),
                 meshgen.box(subdiv=2), TINY["ruff"](), TINY["box_union4"](), TINY["dense_cluster"]()):
        soup = mesh.soup(seed=1)
        feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
        om = oracle.OracleMesh.from_soup(soup)
        assert feats.n_vert == om.V and feats.n_edge == om.E
        assert feats.counts[2:6] == [om.n_convex, om.n_concave, om.n_flat, om.n_saddle]
        assert feats.counts[6:8] == [om.n_convex_edges, om.n_concave_edges]
        vm = feats.vertex_map().cpu().numpy()
        X = feats.vertices().cpu().numpy()
        assert np.array_equal(X[vm], soup.reshape(-1, 3))


def test_build_errors():
    soup = meshgen.icosphere(3).soup(seed=1)
    def code(s):
        with pytest.raises(sdf.SDFError) as e:
            sdf.sdf_build_features(torch.from_numpy(np.ascontiguousarray(s)).cuda())
        return e.value.code
    assert code(soup[1:]) == 2                     # open surface
    fl = soup.copy(); fl[0] = fl[0][[0, 2, 1]]
    assert code(fl) == 2                           # one flipped face
    bad = soup.copy(); bad[4, 1, 0] = np.nan
    assert code(bad) == 4                          # non-finite
    deg = soup.copy(); deg[6, 2] = deg[6, 1]
    assert code(deg) in (2, 3)                     # zero-area / zero-length


def test_empty_band_and_tiny_grid():
    soup = meshgen.icosphere(2, radius=0.1, center=(3.0, 3.0, 3.0)).soup(seed=1)
    feats, (dist, win) = gpu_band(soup, sdf.Grid.cube(40), 3 / 40, winner=True)
    assert torch.all(dist == float("inf")) and torch.all(win == -1)
    soup = meshgen.icosphere(2, radius=0.3).soup(seed=1)
    full_grid_case(soup, sdf.Grid(1, 1, 1, (f32(0.2), 0.2, 0.2), 0.1), 0.2)
    full_grid_case(soup, sdf.Grid(3, 5, 2, (0.0, 0.0, 0.0), 0.25), 0.4)


def test_deterministic_bitwise():
    soup = meshgen.config_soup(1)
    _, (d1, w1) = gpu_band(soup, sdf.Grid.cube(64), 3 / 64, winner=True)
    _, (d2, w2) = gpu_band(soup, sdf.Grid.cube(64), 3 / 64, winner=True)
    assert torch.equal(d1, d2) and torch.equal(w1, w2)


def test_batch_equals_single_calls():
    soups = [meshgen.config_soup(1), TINY["torus_small"]().soup(seed=2), TINY["saddle"]().soup(seed=3)]
    grids = [sdf.Grid.cube(64), sdf.Grid(50, 40, 30, (0.1, 0.1, 0.3), f32(0.0151)), sdf.Grid.cube(32)]
    ws = [3 / 64, f32(3 * 0.0151), 3 / 32]
    feats = [sdf.sdf_build_features(torch.from_numpy(s).cuda()) for s in soups]
    batch = sdf.sdf_narrow_band(feats, grids, ws)
    for f, g, w, b in zip(feats, grids, ws, batch):
        single = sdf.sdf_narrow_band(f, g, w)
        assert torch.equal(single, b)


def test_update_positions_matches_oracle_and_fresh_build():
    m0 = meshgen.icosphere(6, radius=0.3, displacement=0.02, seed=1)
    m1 = meshgen.icosphere(6, radius=0.3, displacement=0.03, seed=2)
    s0 = m0.soup(seed=5)
    feats = sdf.sdf_build_features(torch.from_numpy(s0).cuda())
    # move the welded vertices to m1's positions (same connectivity, same soup order)
    s1 = meshgen.Mesh(m1.vertices, m0.triangles).soup(seed=5)
    vm = feats.vertex_map().cpu().numpy()
    X1 = np.zeros((feats.n_vert, 3), dtype=np.float32)
    X1[vm] = s1.reshape(-1, 3)
    feats.update_positions(torch.from_numpy(X1).cuda())
    grid, w = sdf.Grid.cube(96), 3 / 96
    d_upd = sdf.sdf_narrow_band(feats, grid, w).cpu().numpy()
    _, ref = oracle_dense(s1, grid, w)
    parity.assert_parity(parity.compare(d_upd, ref, w, grid.h))
    # a fresh build numbers vertices and edges differently (Morton order of the new positions), so
    # values may differ by FP32 rounding only
    fresh = sdf.sdf_build_features(torch.from_numpy(s1).cuda())
    d_new = sdf.sdf_narrow_band(fresh, grid, w).cpu().numpy()
    fin = np.isfinite(d_new) & np.isfinite(d_upd)
    assert np.max(np.abs(d_new[fin] - d_upd[fin])) <= 1e-6
    assert fresh.counts == feats.counts


def test_saddle_ablation_leaves_gaps():
    # negative control (Section 11.1, Fig. ear): without saddle extrusions the band has holes
    soup = meshgen.torus(nu=80, nv=32, seed=3).soup(seed=1)
    grid, w = sdf.Grid.cube(96), 3 / 96
    _, d_ok = gpu_band(soup, grid, w)
    _, d_abl = gpu_band(soup, grid, w, flags=sdf.FLAG_DISABLE_SADDLE)
    om, ref = oracle_dense(soup, grid, w)
    st_ok = parity.compare(d_ok.cpu().numpy(), ref, w, grid.h)
    st_abl = parity.compare(d_abl.cpu().numpy(), ref, w, grid.h)
    parity.assert_parity(st_ok)
    assert st_abl["missing"] + st_abl["max_abs_err"] > 0 and (st_abl["missing"] > 0 or st_abl["max_abs_err"] > 1e-4)


def _sampled_case(index: int, n_samples: int, seed: int):
    soup = meshgen.config_soup(index)
    N, cells = meshgen.CONFIG_GRID[index]
    grid, w = sdf.Grid.cube(N), cells / N
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    dist = sdf.sdf_narrow_band(feats, grid, w)
    idx = parity.near_surface_indices(soup, (N, N, N), (0, 0, 0), grid.h, w, n_samples, seed,
                                      n_uniform=n_samples // 10)
    d_gpu = dist.view(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    om = oracle.OracleMesh.from_soup(soup)
    d_or, _, _ = om.band_points((N, N, N), (0, 0, 0), grid.h, w + 2 * grid.h, idx)
    st = parity.compare(d_gpu, d_or, w, grid.h)
    parity.assert_parity(st)
    stat = feats.status()
    band_total = int(torch.isfinite(dist).sum())
    # the tile kernel counts its FP32 decisions; the FP64 re-decision may move only queued points
    assert abs(stat["band_points"] - band_total) <= stat["fp64_points"]
    stat["band_total"] = band_total
    del dist
    torch.cuda.empty_cache()
    return st, stat


def test_c2_torus_sampled():
    st, stat = _sampled_case(2, 60_000, 353_202)
    print(st, stat)


def test_c5_icosphere_sampled():
    st, stat = _sampled_case(5, 40_000, 353_205)
    print(st, stat)


def test_c4_knot_tube_sampled():
    st, stat = _sampled_case(4, 200_000, 353_204)
    print(st, stat)


def test_adjoint_matches_oracle_adjoint():
    for soup, N in ((meshgen.config_soup(1), 64), (TINY["torus_small"]().soup(seed=9), 96)):
        grid, w = sdf.Grid.cube(N), 3 / N
        feats, (dist, win) = gpu_band(soup, grid, w, winner=True)
        rng = np.random.default_rng(1)
        g = torch.from_numpy(rng.normal(size=grid.shape).astype(np.float32)).cuda()
        g = torch.where(torch.isfinite(dist), g, torch.zeros_like(g))
        gv = sdf.sdf_narrow_band_backward(feats, grid, w, g, winner=win)
        gv2 = sdf.sdf_narrow_band_backward(feats, grid, w, g, winner=None)  # recomputed winners
        torch.cuda.synchronize()
        # same winners, different atomicAdd order: equal up to FP32 summation rounding
        assert float((gv - gv2).norm()) <= 1e-5 * float(gv.norm())
        band = torch.isfinite(dist).view(-1).cpu().numpy()
        idx = np.flatnonzero(band)
        pts = oracle.grid_points((N, N, N), (0, 0, 0), grid.h, idx)
        om = oracle.OracleMesh.from_soup(soup)
        go = om.adjoint_points(pts, g.view(-1).cpu().numpy()[idx].astype(np.float64), w + 1e-9)
        a = gv.cpu().numpy()[feats.vertex_map().cpu().numpy()]
        b = go[om.soup_vid()]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel < 1e-3, rel


def test_pair_list_overflow_is_retried(monkeypatch):
    """Few large triangles on a fine grid, with the first (tile, region) pair capacity forced below
    what the binning needs (SDF_PAIR_CAPACITY): the first launch overflows, and the call grows the
    list and runs again."""
    soup = meshgen.config_soup(1)  # 320 triangles, each about 50 cells wide at 512^3
    N = 384
    grid, w = sdf.Grid.cube(N), 3 / N
    monkeypatch.setenv("SDF_PAIR_CAPACITY", "1000")
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    dist = sdf.sdf_narrow_band(feats, grid, w)
    st = feats.status()
    assert st["pairs"] > 1000  # beyond the first capacity
    monkeypatch.delenv("SDF_PAIR_CAPACITY")
    feats2 = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    assert torch.equal(sdf.sdf_narrow_band(feats2, grid, w), dist)
    idx = parity.near_surface_indices(soup, (N, N, N), (0, 0, 0), grid.h, w, 20_000, 353_384, n_uniform=2000)
    d_gpu = dist.view(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    om = oracle.OracleMesh.from_soup(soup)
    d_or, _, _ = om.band_points((N, N, N), (0, 0, 0), grid.h, w + 2 * grid.h, idx)
    parity.assert_parity(parity.compare(d_gpu, d_or, w, grid.h))


@pytest.mark.parametrize("N", [256, 512])
def test_unsynchronised_call_on_a_fresh_handle_has_room(N):
    """A call that does not synchronise cannot grow its scratch and repeat, so a fresh handle's
    first capacity must hold the (tile, region) pairs of large triangles on a fine grid: it comes
    from the build's face-box moments, and it needs to exceed the old 8-per-feature floor here."""
    soup = meshgen.config_soup(1)
    grid, w = sdf.Grid.cube(N), 3 / N
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    dist = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
    sdf.sdf_narrow_band(feats, grid, w, out=dist, flags=sdf.FLAG_NO_SYNC)
    st = feats.status()  # raises on an overflow
    if N == 512:
        assert st["pairs"] > 8 * (feats.n_tri + feats.n_edge + feats.n_vert) + 4096
    ref = sdf.sdf_narrow_band(sdf.sdf_build_features(torch.from_numpy(soup).cuda()), grid, w)
    assert torch.equal(dist, ref)


def test_split_tiles_agree_bitwise_with_unsplit_paths():
    """A densely subdivided part puts about 250 k regions into a few tiles, which the tile kernel
    splits over many CTAs (their keys merged with atomicMin in global memory, the last item decoding
    the tile).  The merge is order-independent, so the field equals bit for bit the allocation-free
    entry point's (which never splits), the band-list call's, and a batch's (split tiles listed in
    largest-first order); the full-grid oracle comparison of the same mesh is
    test_small_meshes_full_grid_dyadic[dense_cluster]."""
    import ctypes
    soup = TINY["dense_cluster"]().soup(seed=5)
    grid, w = sdf.Grid.cube(96), 3 / 96
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    dist, win = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    st = feats.status()
    assert st["pairs"] > 100_000
    d_static = torch.empty_like(dist)
    w_static = torch.empty_like(win)
    L = sdf.load_library()
    cg = grid.c()
    assert L.sdf_narrow_band_static(feats.handle, ctypes.byref(cg), ctypes.c_float(w), d_static.data_ptr(),
                                    w_static.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    assert torch.equal(dist, d_static) and torch.equal(win, w_static)
    d_list, bl = sdf.sdf_narrow_band_list(feats, grid, w)
    assert torch.equal(dist, d_list)
    other = sdf.sdf_build_features(torch.from_numpy(meshgen.icosphere(6, radius=0.3).soup(seed=6)).cuda())
    b = sdf.sdf_batch_create([other, feats], [sdf.Grid.cube(64), grid], [3 / 64, w])
    b.run()
    torch.cuda.synchronize()
    assert torch.equal(b.outs[1], dist)
    assert torch.equal(b.outs[0], sdf.sdf_narrow_band(other, sdf.Grid.cube(64), 3 / 64))
    b.destroy()
