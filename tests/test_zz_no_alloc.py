"""The allocation-free narrow band (sdf_narrow_band_static), called through the C ABI.

Some callers cannot allocate device memory while they run (their memory belongs to another
runtime or a fixed budget, or they cannot afford an allocation's latency).  For them the
library offers one entry point whose scratch is a fixed device array inside the library.  This
test checks, on two calls in a row (the second one finds the first one's leftovers in the
shared array), that it returns the same field and winners as the regular sdf_narrow_band,
within the tolerance of the parity tests, that those calls take no device memory from the
library's pool and no pinned host memory, that a grid beyond the array's limit is rejected, and
that positions which collapse a face are reported as the regular call reports them.  It lives in
its own file, collected last, and passes alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1903_00353_gb300 as sdf
    return sdf


def _static_call(sdf, feats, grid, w, dist, win):
    L = sdf.load_library()
    cg = grid.c()
    return L.sdf_narrow_band_static(feats.handle, ctypes.byref(cg), ctypes.c_float(w), dist.data_ptr(),
                                    win.data_ptr() if win is not None else None,
                                    torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("case", ["icosphere_64", "torus_ragged"])
def test_static_matches_regular_two_calls(lib, case):
    sdf = lib
    if case == "icosphere_64":
        soup = meshgen.config_soup(1)
        grid, w = sdf.Grid.cube(64), 3 / 64
    else:
        soup = meshgen.torus(nu=60, nv=24, seed=3).soup(seed=2)
        h = float(np.float32(0.0123))
        grid, w = sdf.Grid(90, 77, 45, (0.0, 0.0, float(np.float32(0.23))), h), float(np.float32(3 * h))
    feats = sdf.sdf_build_features(torch.from_numpy(soup).cuda())
    ref_d, ref_w = sdf.sdf_narrow_band(feats, grid, w, winner=True)
    outs = [(torch.full(grid.shape, 7.0, dtype=torch.float32, device="cuda"),
             torch.full(grid.shape, -7, dtype=torch.int32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    before = sdf.memory_stats()
    torch_before = torch.cuda.memory_allocated()
    for d, wn in outs:
        assert _static_call(sdf, feats, grid, w, d, wn) == 0
    torch.cuda.synchronize()
    after = sdf.memory_stats()
    # no allocation of any kind during the two calls: none from the library's device pool (count,
    # bytes in use and reserved unchanged), no pinned host block, nothing through torch
    assert after == before, (before, after)
    assert torch.cuda.memory_allocated() == torch_before
    fin = torch.isfinite(ref_d)
    for d, wn in outs:
        assert torch.equal(fin, torch.isfinite(d))
        assert float((d[fin] - ref_d[fin]).abs().max()) <= 2e-6
        assert torch.equal(wn, ref_w)


def test_static_rejects_grid_beyond_limit(lib):
    sdf = lib
    feats = sdf.sdf_build_features(torch.from_numpy(meshgen.config_soup(1)).cuda())
    grid = sdf.Grid(1024, 1024, 16, (0.0, 0.0, 0.5), 1 / 1024)  # 32 * 128 * 2 = 8192 tiles: fits
    d = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
    assert _static_call(sdf, feats, grid, 3 / 1024, d, None) == 0
    big = sdf.Grid(1024, 1024, 600, (0.0, 0.0, 0.0), 1 / 1024)  # 32 * 128 * 75 tiles > 65536
    assert _static_call(sdf, feats, big, 3 / 1024, d, None) == 5  # SDF_ERR_TOO_LARGE, before any work


def test_static_reports_a_collapsed_face(lib):
    """Positions that collapse a face (one corner moved onto another): both the regular and the
    allocation-free call return SDF_ERR_DEGENERATE (3)."""
    sdf = lib
    feats = sdf.sdf_build_features(torch.from_numpy(meshgen.icosphere(3, radius=0.3).soup(seed=4)).cuda())
    grid, w = sdf.Grid.cube(48), 3 / 48
    X = feats.vertices().clone()
    tri = feats.vertex_map().view(-1, 3)[0].tolist()
    X[tri[1]] = X[tri[0]]
    feats.update_positions(X)
    d = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
    assert _static_call(sdf, feats, grid, w, d, None) == 3
    with pytest.raises(sdf.SDFError) as e:
        sdf.sdf_narrow_band(feats, grid, w, out=d)
    assert e.value.code == 3
