"""FLAG_TIMING on a features handle: the events of timed calls are read later (by the next timed
call or by Features.timing), never by the call itself; every timed call is counted once, with a
positive time per stage, and reset clears the totals.  GPU only."""
import pytest
import torch

import meshgen
import paper_1903_00353_gb300 as sdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_timed_calls_are_counted_once_each():
    feats = sdf.sdf_build_features(torch.from_numpy(meshgen.config_soup(1)).cuda())
    grid, w = sdf.Grid.cube(64), 3 / 64
    assert all(c == 0 for _, c in feats.timing().values())
    d0 = sdf.sdf_narrow_band(feats, grid, w, flags=sdf.FLAG_TIMING | sdf.FLAG_NO_SYNC)
    d1, bl = sdf.sdf_narrow_band_list(feats, grid, w, flags=sdf.FLAG_TIMING)
    g = torch.where(torch.isfinite(d1), torch.ones_like(d1), torch.zeros_like(d1))
    sdf.band_list_backward(feats, grid, bl, g, flags=sdf.FLAG_TIMING)
    t = feats.timing(reset=True)
    for stage in ("bin", "tile", "fp64"):
        ms, calls = t[stage]
        assert calls == 2 and ms > 0.0, (stage, t)
    assert t["adjoint"][1] == 1 and t["adjoint"][0] > 0.0
    assert torch.equal(d0, d1)
    assert all(c == 0 for _, c in feats.timing().values())
    # untimed calls add nothing
    sdf.sdf_narrow_band(feats, grid, w)
    assert all(c == 0 for _, c in feats.timing().values())
    feats.destroy()
