"""The build's sorts in one cooperative launch against three launches per pass, through the C ABI.

sdf_build_features sorts the soup's corners by their weld key (40 bits, five 8-bit passes) and the
faces by their smallest vertex id (Section 7).  A sort whose tiles all fit on the GPU at once runs
every pass in one cooperative launch, with grid barriers between its phases; the environment
variable SDF_RADIX_ONE_LAUNCH=0 keeps the three launches per pass (digit histograms, their scan,
the scatter).  Both are stable LSD radix sorts of the same keys, so the welded vertex ids, the face
order, the edge table, the field and the winners must agree bitwise, and the one-launch build must
make exactly 3P - 1 fewer launches for each sort of P passes.  The cases span the three tile sizes
(2, 4 and 8 keys per thread) and long runs of equal weld keys.  GPU only.
"""
import numpy as np
import pytest
import torch

import meshgen
import paper_1903_00353_gb300 as sdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


CASES = {
    "icosphere_c1": lambda: meshgen.config_soup(1),
    "torus_50k": lambda: meshgen.config_soup(2),                 # 150 k corners: 2 keys per thread
    "torus_80k": lambda: meshgen.torus(nu=250, nv=160, seed=5).soup(seed=4),  # 240 k corners: 4
    "icosphere_200k": lambda: meshgen.config_soup(5),            # 600 k corners: 8
    "dense_cluster": lambda: meshgen.dense_cluster().soup(seed=1),  # long runs of equal weld keys
}


def _build(soup_t, monkeypatch, one_launch: bool):
    if one_launch:
        monkeypatch.delenv("SDF_RADIX_ONE_LAUNCH", raising=False)
    else:
        monkeypatch.setenv("SDF_RADIX_ONE_LAUNCH", "0")
    torch.cuda.synchronize()
    l0 = sdf.kernel_launches()
    feats = sdf.sdf_build_features(soup_t)
    torch.cuda.synchronize()
    return feats, sdf.kernel_launches() - l0


def _passes(bits: int) -> int:
    return (bits + 7) // 8


@pytest.mark.parametrize("case", list(CASES))
def test_one_launch_sort_agrees_with_launches_per_pass(case, monkeypatch):
    soup = CASES[case]()
    soup_t = torch.from_numpy(np.ascontiguousarray(soup, dtype=np.float32)).cuda()
    f_one, n_one = _build(soup_t, monkeypatch, True)
    f_pass, n_pass = _build(soup_t, monkeypatch, False)
    assert f_one.counts == f_pass.counts
    assert torch.equal(f_one.vertex_map(), f_pass.vertex_map())
    assert torch.equal(f_one.face_map(), f_pass.face_map())
    assert torch.equal(f_one.edges(), f_pass.edges())
    assert torch.equal(f_one.vertices(), f_pass.vertices())
    # the face sort's key holds the bits of the largest vertex id
    face_bits = 1
    while (1 << face_bits) < f_one.n_vert:
        face_bits += 1
    expect = (3 * _passes(40) - 1) + (3 * _passes(face_bits) - 1)
    assert n_pass - n_one == expect, (n_pass, n_one, expect)
    grid, w = sdf.Grid.cube(128), 3.0 / 128
    d1, w1 = sdf.sdf_narrow_band(f_one, grid, w, winner=True)
    d2, w2 = sdf.sdf_narrow_band(f_pass, grid, w, winner=True)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)
    assert torch.equal(w1, w2)
    assert int(torch.isfinite(d1).sum()) > 0
