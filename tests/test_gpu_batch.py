"""Batches of (mesh, grid) problems in one launch sequence: equality with the single-problem path,
replay (plain and inside a CUDA graph), tile-shape autotuning, and parity with the FP64 oracle on
a mixed batch that includes clusters of rotated boxes.  GPU only."""
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


def _problems():
    """Uneven meshes on ragged, non-cubic grids: a displaced icosphere, a torus, a box cluster,
    a saddle solid, a small knot tube and a union of overlapping boxes."""
    meshes = [meshgen.icosphere(8, radius=0.3, displacement=0.02, seed=11),
              meshgen.torus(nu=60, nv=24, seed=12),
              meshgen.box_cluster(3, 3000, seed=13),
              meshgen.star_fan_solid(8, [0.06, -0.06] * 4, apex_h=0.0),
              meshgen.knot_tube(n_along=600, n_around=12, seed=14),
              meshgen.box_union(3, 2500, seed=15)]
    grids = [sdf.Grid.cube(64),
             sdf.Grid(70, 45, 38, (0.05, 0.12, 0.21), f32(0.0201)),
             sdf.Grid.cube(96),
             sdf.Grid(33, 64, 17, (0.1, 0.0, 0.35), f32(1 / 60)),
             sdf.Grid(100, 100, 40, (0.0, 0.0, 0.3), f32(0.01)),
             sdf.Grid(61, 70, 66, (0.02, 0.01, 0.03), f32(0.0141))]
    ws = [3 * g.h for g in grids]
    soups = [m.soup(seed=20 + i) for i, m in enumerate(meshes)]
    feats = [sdf.sdf_build_features(torch.from_numpy(s).cuda()) for s in soups]
    return soups, feats, grids, ws


def _singles(feats, grids, ws):
    out = []
    for f, g, w in zip(feats, grids, ws):
        d, wn = sdf.sdf_narrow_band(f, g, w, winner=True)
        out.append((d.clone(), wn.clone()))
    return out


def _garbage(batch):
    for o in batch.outs:
        o.fill_(-123.0)
    for wn in batch.winners:
        wn.fill_(-7)


def _assert_equal(batch, singles):
    for (d, wn), o, bw in zip(singles, batch.outs, batch.winners):
        assert torch.equal(d, o)
        assert torch.equal(wn, bw)


def test_batch_create_run_equals_single_calls():
    soups, feats, grids, ws = _problems()
    singles = _singles(feats, grids, ws)
    batch = sdf.sdf_batch_create(feats, grids, ws, winner=True)
    torch.cuda.synchronize()
    _assert_equal(batch, singles)
    assert batch.info()["tile"] == (32, 8, 8)
    for _ in range(2):
        _garbage(batch)
        batch.run()
        torch.cuda.synchronize()
        _assert_equal(batch, singles)
    st = batch.status()
    assert st["band_points"] > 0 and st["candidates"] >= st["band_points"]
    with pytest.raises(sdf.SDFError):
        batch.timing()  # created without timing
    batch.destroy()


def test_batch_replays_inside_cuda_graph():
    soups, feats, grids, ws = _problems()
    singles = _singles(feats, grids, ws)
    batch = sdf.sdf_batch_create(feats, grids, ws, winner=True, timing=True)
    torch.cuda.synchronize()
    launches0 = sdf.kernel_launches()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            batch.run()
    torch.cuda.synchronize()
    captured = sdf.kernel_launches() - launches0
    assert captured >= 6  # bin x2, scans, flags, lists, tile, patch recorded into the graph
    for _ in range(3):
        _garbage(batch)
        graph.replay()
        torch.cuda.synchronize()
        _assert_equal(batch, singles)
        t = batch.timing()  # the event nodes of the replay
        assert t["bin"] > 0.0 and t["tile"] > 0.0 and t["fp64"] > 0.0
    # launches are counted when enqueued: replays add none
    assert sdf.kernel_launches() - launches0 == captured
    assert batch.status()["band_points"] > 0
    del graph
    batch.destroy()


def test_batch_follows_position_updates():
    soups, feats, grids, ws = _problems()
    batch = sdf.sdf_batch_create(feats[:2], grids[:2], ws[:2], winner=True)
    X = feats[0].vertices()
    X2 = (X - 0.5) * 1.03 + 0.5  # scale the icosphere about the centre by 3 %
    feats[0].update_positions(X2.contiguous())
    batch.run()
    torch.cuda.synchronize()
    d, wn = sdf.sdf_narrow_band(feats[0], grids[0], ws[0], winner=True)
    assert torch.equal(d, batch.outs[0]) and torch.equal(wn, batch.winners[0])
    d1, wn1 = sdf.sdf_narrow_band(feats[1], grids[1], ws[1], winner=True)
    assert torch.equal(d1, batch.outs[1])
    batch.destroy()


def test_autotuned_batch_matches_oracle():
    soups, feats, grids, ws = _problems()
    batch = sdf.sdf_batch_create(feats, grids, ws, winner=True, autotune=True)
    torch.cuda.synchronize()
    info = batch.info()
    assert info["tile"] in {(32, 8, 8), (32, 4, 4), (32, 16, 8)}
    assert info["tuned_ms"] > 0.0
    for soup, g, w, o, f, wn in zip(soups, grids, ws, batch.outs, feats, batch.winners):
        om = oracle.OracleMesh.from_soup(soup)
        ref = om.narrow_band((g.nx, g.ny, g.nz), g.origin, g.h, w + 2 * g.h)
        st = parity.compare(o.cpu().numpy(), ref, w, g.h)
        parity.assert_parity(st)
        assert st["band_oracle"] > 0
        band = torch.isfinite(o)
        n_feat = f.n_tri + f.n_edge + f.n_vert
        assert bool((wn[~band] == -1).all()) and bool(((wn[band] >= 0) & (wn[band] < n_feat)).all())
    # the replay of an autotuned batch reproduces its own first result bit for bit
    first = [o.clone() for o in batch.outs]
    _garbage(batch)
    batch.run()
    torch.cuda.synchronize()
    for a, b in zip(first, batch.outs):
        assert torch.equal(a, b)
    batch.destroy()


def test_list_call_uses_tuned_shape_and_matches_oracle():
    """sdf_narrow_band with n > 1 after autotuning the same sizes runs with the remembered shape."""
    soups, feats, grids, ws = _problems()
    batch = sdf.sdf_batch_create(feats, grids, ws, autotune=True)
    torch.cuda.synchronize()
    res = sdf.sdf_narrow_band(feats, grids, ws)
    for a, b in zip(batch.outs, res):
        assert torch.equal(a, b)
    batch.destroy()


def test_batch_argument_errors():
    soups, feats, grids, ws = _problems()
    with pytest.raises(ValueError):
        sdf.sdf_batch_create(feats[:2], grids[:1], ws[:2])
    with pytest.raises(sdf.SDFError):
        sdf.sdf_batch_create(feats[:1], grids[:1], [0.0])
    bad = sdf.Grid(0, 4, 4, (0.0, 0.0, 0.0), 0.1)
    with pytest.raises((sdf.SDFError, ValueError, RuntimeError)):
        sdf.sdf_batch_create(feats[:1], [bad], [0.1], out=[torch.empty(1, device="cuda")])
