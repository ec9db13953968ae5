"""Checks of the synthetic input meshes: closed, oriented 2-manifolds with the sizes the
workloads name, no degenerate triangles, the expected Euler characteristic, and exact
duplicate coordinates in the soup (Section 7 reading of "identical" vertices)."""
import numpy as np
import pytest

import meshgen


def _check_closed_oriented(mesh: meshgen.Mesh):
    tri = mesh.triangles.astype(np.int64)
    a = tri.ravel()
    b = tri[:, [1, 2, 0]].ravel()
    directed = set(zip(a.tolist(), b.tolist()))
    assert len(directed) == a.size, "a directed edge appears twice (not oriented)"
    for u, v in directed:
        assert (v, u) in directed, "open edge"
    X = mesh.vertices
    cr = np.cross(X[tri[:, 1]] - X[tri[:, 0]], X[tri[:, 2]] - X[tri[:, 0]])
    area2 = np.linalg.norm(cr, axis=1)
    assert area2.min() > 1e-12
    vol = np.einsum("ij,ij->i", X[tri[:, 0]], np.cross(X[tri[:, 1]], X[tri[:, 2]])).sum() / 6
    assert vol > 0
    return len(directed) // 2


@pytest.mark.parametrize("freq", [1, 2, 4, 7])
def test_icosphere_counts(freq):
    m = meshgen.icosphere(freq)
    assert m.triangles.shape[0] == 20 * freq * freq
    assert m.vertices.shape[0] == 10 * freq * freq + 2
    E = _check_closed_oriented(m)
    assert m.vertices.shape[0] - E + m.triangles.shape[0] == 2


def test_config1_sizes():
    m = meshgen.config_mesh(1)
    assert m.triangles.shape == (320, 3) and m.vertices.shape == (162, 3)
    r = np.linalg.norm(m.vertices - 0.5, axis=1)
    assert np.allclose(r, 0.3)


def test_torus_small_and_config2_sizes():
    m = meshgen.torus(nu=30, nv=12, seed=1)
    E = _check_closed_oriented(m)
    assert m.vertices.shape[0] - E + m.triangles.shape[0] == 0
    m2 = meshgen.config_mesh(2)
    assert m2.triangles.shape[0] == 50_000 and m2.vertices.shape[0] == 25_000


def test_knot_tube_small():
    m = meshgen.knot_tube(n_along=512, n_around=16, seed=3)
    E = _check_closed_oriented(m)
    assert m.vertices.shape[0] - E + m.triangles.shape[0] == 0


def test_knot_strand_separation():
    # strands must stay far apart compared with 2*(tube radius + noise) + 2*band
    sep = meshgen.knot_min_strand_separation()
    assert sep > 2 * 0.045 + 2 * 3 / 1024 + 0.02, sep


def test_soup_duplicates_are_bitwise_equal():
    m = meshgen.icosphere(3, displacement=0.02, seed=5)
    s = m.soup(seed=9)
    flat = s.reshape(-1, 3)
    uniq = np.unique(flat.view(np.dtype((np.void, 12))))
    assert uniq.shape[0] == m.vertices.shape[0]


def test_soup_shuffle_preserves_orientation():
    m = meshgen.icosphere(2)
    s = m.soup(seed=1).astype(np.float64)
    n = np.cross(s[:, 1] - s[:, 0], s[:, 2] - s[:, 0])
    c = s.mean(axis=1) - 0.5
    assert np.all(np.einsum("ij,ij->i", n, c) > 0)


def test_box_and_tetra_closed():
    for m in (meshgen.box(subdiv=2), meshgen.regular_tetrahedron(), meshgen.octahedron(),
              meshgen.star_fan_solid(8, [0.05, -0.05] * 4)):
        E = _check_closed_oriented(m)
        assert m.vertices.shape[0] - E + m.triangles.shape[0] == 2


def test_batch_meshes_sizes():
    batch = meshgen.batch_meshes(n=8, t_max=2e4)
    for mesh, N in batch:
        _check_closed_oriented(mesh)
        assert 64 <= N <= 384 and N % 32 == 0


@pytest.mark.parametrize("k", [2, 3, 4])
def test_box_cluster_components(k):
    m = meshgen.box_cluster(k, 2000, seed=353_300 + k)
    E = _check_closed_oriented(m)
    # k disjoint spheres: Euler characteristic 2 per component
    assert m.vertices.shape[0] - E + m.triangles.shape[0] == 2 * k
    assert m.vertices.min() > 0.0 and m.vertices.max() < 1.0


def test_random_rotation_is_proper():
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(10):
        R = meshgen.random_rotation(rng)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12


def _box_halfspaces(c, R, half):
    """The box c + R diag(half) [-1, 1]^3 as rows [n, -d] of n.x - d <= 0 (scipy's convention)."""
    rows = []
    for k in range(3):
        for s in (-1.0, 1.0):
            n = s * R[:, k]
            rows.append(np.concatenate([n, [-(n @ c + half[k])]]))
    return np.array(rows)


def _convex_volume(H):
    """Volume of the polytope {x : H[:, :3] x + H[:, 3] <= 0}, 0 if it has no interior: an interior
    point from the Chebyshev-centre linear programme, the vertices from qhull's halfspace
    intersection, the volume from their convex hull."""
    from scipy.optimize import linprog
    from scipy.spatial import ConvexHull, HalfspaceIntersection
    A, b = H[:, :3], -H[:, 3]
    norm = np.linalg.norm(A, axis=1)
    res = linprog([0, 0, 0, -1], A_ub=np.hstack([A, norm[:, None]]), b_ub=b, bounds=[(None, None)] * 3 + [(0, None)])
    if res.status != 0 or res.x[3] < 1e-9:
        return 0.0
    hs = HalfspaceIntersection(H, res.x[:3])
    return ConvexHull(hs.intersections).volume


@pytest.mark.parametrize("k", [2, 3, 4])
def test_box_union_is_the_union_boundary(k):
    """The union mesh is closed and oriented, every vertex lies on some box's surface and inside
    none, and its enclosed volume equals the union's volume by inclusion-exclusion over the boxes'
    intersections (convex polytopes measured with qhull, independent of the face clipping)."""
    import itertools
    m, boxes = meshgen.box_union(k, 2000, seed=353_310 + k, return_boxes=True)
    E = _check_closed_oriented(m)
    T, V = m.triangles.shape[0], m.vertices.shape[0]
    assert V - E + T == 2
    assert 2000 / 2.1 <= T <= 2000 * 2.1
    assert m.vertices.min() > 0.05 - 1e-12 and m.vertices.max() < 0.95 + 1e-12
    sd = np.stack([_box_sdf_rotated(m.vertices, *b) for b in boxes])
    assert np.abs(sd).min(axis=0).max() < 1e-12
    assert sd.min(axis=0).min() > -1e-12
    H = [_box_halfspaces(*b) for b in boxes]
    vol_union = 0.0
    for r in range(1, k + 1):
        for sub in itertools.combinations(range(k), r):
            vol_union += (-1) ** (r + 1) * _convex_volume(np.concatenate([H[i] for i in sub]))
    X, tri = m.vertices, m.triangles
    vol_mesh = np.einsum("ij,ij->i", X[tri[:, 0]], np.cross(X[tri[:, 1]], X[tri[:, 2]])).sum() / 6
    assert abs(vol_mesh - vol_union) < 1e-12 * max(1.0, vol_union) * 100
    # the boxes overlap: the union is smaller than the sum of the boxes
    assert vol_union < sum(8 * np.prod(b[2]) for b in boxes) - 1e-6


def _box_sdf_rotated(p, c, R, half):
    """Exact SDF of the box c + R diag(half) [-1, 1]^3 (in the box's frame: |max(q,0)| + min(max q, 0))."""
    q = np.abs((np.asarray(p) - c) @ R) - half
    return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(q.max(axis=-1), 0.0)


def test_box_union_is_seeded():
    a = meshgen.box_union(3, 1500, seed=5)
    b = meshgen.box_union(3, 1500, seed=5)
    assert np.array_equal(a.vertices, b.vertices) and np.array_equal(a.triangles, b.triangles)
