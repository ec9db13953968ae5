"""Parity at the full sizes of the workloads, through the C ABI, against the FP64 oracle (GPU only).

  * the vertex adjoint on the 50k-triangle torus at 512^3 (band 4h) and on the 200k-triangle
    icosphere at steps 0, 10 and 19 of the 20-step shape fit (512^3, band 4h), each checked two
    ways: against the oracle's adjoint evaluated on the GPU's own winners (the features' FP64
    closest points: isolates the FP32 arithmetic, relative L2 <= 1e-5) and against the oracle's
    adjoint with its own winners (relative L2 <= 1e-3; the difference comes from near ties,
    which are counted);
  * the 2.1M-triangle knot tube at 1024^3 (band 3h) on 10^6 points, stratified: every grid point
    whose FP32 value lies within 2 delta of the band edge or of the surface (all of them; the
    grid holds only a few tens of thousands), topped up to 10^5 with points within 20 delta, and
    the rest drawn near the surface and uniformly over the mesh's box;
  * the 64-problem batch (1e3..2e5 triangles, grids 64^3..384^3, band 3h): bitwise equal to the
    64 single calls with the same tile shape, the autotuned batch within the tolerance, and 10^4
    oracle samples per mesh.
"""
import numpy as np
import pytest
import torch

import meshgen
import oracle
import paper_1903_00353_gb300 as sdf
from tests import parity

pytestmark = pytest.mark.gpu

ADJ_OWN_WINNERS = 1e-5   # GPU FP32 adjoint vs the FP64 adjoint on the GPU's winners
ADJ_ORACLE = 1e-3        # vs the oracle's own winners (near ties)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _adjoint_two_ways(feats, grid, w, dist, win, g_dense, label):
    """GPU adjoint (FP64 accumulation of the FP32 contributions) against the oracle on the GPU's
    winners and on its own."""
    N = grid.nx
    gv = torch.zeros(feats.n_vert, 3, dtype=torch.float64, device="cuda")
    sdf.sdf_narrow_band_backward(feats, grid, w, g_dense, winner=win, grad_vertices=gv)
    torch.cuda.synchronize()
    a = gv.cpu().numpy()
    band = torch.isfinite(dist).view(-1)
    idx = torch.nonzero(band).view(-1)
    wid = win.view(-1)[idx].cpu().numpy()
    g = g_dense.view(-1)[idx].cpu().numpy().astype(np.float64)
    idx = idx.cpu().numpy()
    pts = oracle.grid_points((grid.nx, grid.ny, grid.nz), grid.origin, grid.h, idx)
    om, wmap = parity.oracle_of_features(feats)
    t, r = wmap(wid)
    b_own, d_own = om.adjoint_features(pts, g, t, r)
    b_or = om.adjoint_points(pts, g, w)
    e_own, e_or = parity.rel_l2(a, b_own), parity.rel_l2(a, b_or)
    # near ties: points whose oracle winner lies on another feature than the GPU's
    d_o, t_o, r_o = om.sdf_points(pts)
    diff = np.abs(np.abs(d_own) - np.abs(d_o))
    ties = int(np.sum(diff > 0))
    print(f"{label}: band {idx.size}, rel L2 vs FP64 on GPU winners {e_own:.2e}, vs oracle winners {e_or:.2e}, "
          f"points where the GPU winner is not an oracle-closest feature {ties} (max gap {diff.max():.2e})")
    assert e_own <= ADJ_OWN_WINNERS, e_own
    assert e_or <= ADJ_ORACLE, e_or
    # the GPU's winners are closest features up to the FP32 error
    assert diff.max() <= feats.error_bound(grid, w)["delta"] * 2
    return e_own, e_or


def test_c2_adjoint_full_band():
    soup = meshgen.config_soup(2)
    N, cells = meshgen.CONFIG_GRID[2]
    grid, w = sdf.Grid.cube(N), cells / N
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    dist, win = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    g = torch.where(torch.isfinite(dist), 2.0 * (dist - 0.01), torch.zeros_like(dist))  # sum_band (d - 0.01)^2
    _adjoint_two_ways(feats, grid, w, dist, win, g, "C2 torus 50k 512^3")
    # the list adjoint (the bench's path) carries the same contributions
    dist2, bl = sdf.sdf_narrow_band_list(feats, grid, w)
    gv_list = torch.zeros(feats.n_vert, 3, dtype=torch.float64, device="cuda")
    sdf.band_list_backward(feats, grid, bl, g, grad_vertices=gv_list)
    gv = torch.zeros(feats.n_vert, 3, dtype=torch.float64, device="cuda")
    sdf.sdf_narrow_band_backward(feats, grid, w, g, winner=win, grad_vertices=gv)
    assert torch.equal(dist2, dist)
    assert float((gv_list - gv).norm()) <= 1e-12 * float(gv.norm())


def test_c5_fit_adjoint_at_steps_0_10_19():
    from bench import FIT_LR, ellipsoid_target
    soup = meshgen.config_soup(5)
    N, cells = meshgen.CONFIG_GRID[5]
    grid, w = sdf.Grid.cube(N), cells / N
    dev = torch.device("cuda")
    target = ellipsoid_target(N, dev)
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    X = feats.vertices().clone()
    dist = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    win = torch.empty(grid.shape, dtype=torch.int32, device=dev)
    losses = []
    for step in range(20):
        feats.update_positions(X)
        sdf.sdf_narrow_band(feats, grid, w, out=dist, winner=win)
        g = torch.where(torch.isfinite(dist), 2.0 * (dist - target), torch.zeros_like(dist))
        losses.append(float(torch.where(torch.isfinite(dist), (dist - target) ** 2, torch.zeros_like(dist))
                            .double().sum()))
        if step in (0, 10, 19):
            _adjoint_two_ways(feats, grid, w, dist, win, g, f"C5 fit step {step}")
        # FP64 sums (order-independent), so that the trajectory is the same on every run
        gv = torch.zeros(feats.n_vert, 3, dtype=torch.float64, device=dev)
        sdf.sdf_narrow_band_backward(feats, grid, w, g, winner=win, grad_vertices=gv)
        X = X - FIT_LR * gv.float()
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.9 * losses[0]


def test_c4_knot_tube_stratified_million():
    soup = meshgen.config_soup(4)
    N, cells = meshgen.CONFIG_GRID[4]
    grid, w = sdf.Grid.cube(N), cells / N
    h = grid.h
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    dist = sdf.sdf_narrow_band(feats, grid, w)
    delta = feats.error_bound(grid, w)["delta"]
    # points near the band edge on both sides come from a second call with a wider band
    wide = sdf.sdf_narrow_band(feats, grid, w + 40 * delta)
    torch.cuda.synchronize()
    a_wide, a = wide.abs(), dist.abs()

    def where(mask):
        return torch.nonzero(mask.view(-1)).view(-1).cpu().numpy()

    edge2 = where((a_wide - w).abs() < 2 * delta)
    surf2 = where(a < 2 * delta)
    within2 = np.union1d(edge2, surf2)
    edge20 = where((a_wide - w).abs() < 20 * delta)
    surf20 = where(a < 20 * delta)
    del wide, a_wide, a
    torch.cuda.empty_cache()
    rng = np.random.default_rng(353_204)
    extra = np.setdiff1d(np.union1d(edge20, surf20), within2)
    n_extra = max(0, min(extra.size, 100_000 - within2.size))
    stratum = np.union1d(within2, rng.choice(extra, size=n_extra, replace=False))
    rest = parity.near_surface_indices(soup, (N, N, N), (0, 0, 0), h, w, 900_000, 353_214, n_uniform=100_000)
    idx = np.union1d(stratum, rest)
    if idx.size > 1_000_000:
        keep = np.setdiff1d(idx, stratum)
        idx = np.union1d(stratum, rng.choice(keep, size=1_000_000 - stratum.size, replace=False))
    om = oracle.OracleMesh.from_soup(soup)
    d_or, _, _ = om.band_points((N, N, N), (0, 0, 0), h, w + 2 * h, idx)
    d_gpu = dist.view(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    st = parity.compare(d_gpu, d_or, w, h)
    near = np.isin(idx, stratum)
    a_or = np.abs(d_or)
    true2 = (np.abs(a_or - w) < 2 * delta) | (a_or < 2 * delta)
    print(f"C4: {idx.size} points, {within2.size} within 2 delta by FP32 (all of the grid's), stratum {stratum.size}, "
          f"oracle-confirmed within 2 delta {int(true2.sum())}, delta {delta:.2e}", st)
    assert idx.size >= 900_000 and stratum.size >= 100_000 and within2.size > 5_000
    if st["sign_mismatch"] or st["mask_mismatch"]:  # diagnostics of the failing points
        g_band, o_band = np.isfinite(d_gpu), np.abs(d_or) < w
        bad = (g_band & o_band & (np.abs(d_or) > 1e-5 * h) & (np.sign(d_gpu) != np.sign(d_or))) | \
              ((g_band != o_band) & (np.abs(a_or - w) > 1e-5 * h))
        win = sdf.sdf_narrow_band(feats, grid, w, winner=True)[1].view(-1)[torch.from_numpy(idx[bad]).cuda()]
        for i, d1, d2, wi in zip(idx[bad][:20], d_gpu[bad][:20], d_or[bad][:20], win.cpu().numpy()[:20]):
            print("mismatch", int(i), float(d1), float(d2), int(wi))
    parity.assert_parity(st)
    assert near.sum() == stratum.size


def _batch_problems():
    return [(m.soup(seed=353_300 + i), N, 3.0 / N) for i, (m, N) in enumerate(meshgen.batch_meshes())]


def test_c3_full_batch():
    problems = _batch_problems()
    assert len(problems) == 64
    feats = [sdf.sdf_build_features(torch.from_numpy(s).cuda()) for s, _, _ in problems]
    grids = [sdf.Grid.cube(N) for _, N, _ in problems]
    ws = [w for _, _, w in problems]
    # one launch for all 64 problems with the default tile shape: bitwise the single calls
    b = sdf.sdf_batch_create(feats, grids, ws)
    tuned = sdf.sdf_batch_create(feats, grids, ws, autotune=True)
    shape = tuned.info()["tile"]
    n_points = 0
    for p, ((soup, N, w), f, g) in enumerate(zip(problems, feats, grids)):
        single = sdf.sdf_narrow_band(f, g, w)
        assert torch.equal(b.outs[p], single), p
        fin = torch.isfinite(single)
        if shape == (32, 8, 8):
            assert torch.equal(tuned.outs[p], single), p
        idx = parity.near_surface_indices(soup, (N, N, N), (0, 0, 0), 1.0 / N, w, 9_000, 353_300 + p,
                                          n_uniform=1_000)
        om = oracle.OracleMesh.from_soup(soup)
        d_or, _, _ = om.band_points((N, N, N), (0, 0, 0), 1.0 / N, w + 2.0 / N, idx)
        it = torch.from_numpy(idx).cuda()
        for out in (b.outs[p], tuned.outs[p]):
            parity.assert_parity(parity.compare(out.view(-1)[it].cpu().numpy(), d_or, w, 1.0 / N))
        n_points += idx.size
        del single, fin
    print("C3: 64 problems, tuned tile", shape, "oracle samples", n_points)
    b.destroy()
    tuned.destroy()
