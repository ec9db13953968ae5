"""Pins of the FP64 CPU oracle against things other than itself (CPU only).

Each test targets a plausible mistake: a dropped term or wrong sign in the
point-triangle distance (exact rationals, closed forms), a wrong pseudonormal or
sign rule (exact ray parity), a wrong pruning bound (literal loop), an index or
layout error (translation / rotation covariance), and a wrong adjoint (finite
differences and exact identities).
"""
import math

import numpy as np
import pytest

import meshgen
import oracle
from tests import exact_ref


def _quantized(mesh: meshgen.Mesh, bits: int = 20) -> meshgen.Mesh:
    """Round vertex coordinates to multiples of 2^-bits (so shifts by k/64 stay exact)."""
    q = np.round(mesh.vertices * (1 << bits)) / (1 << bits)
    return meshgen.Mesh(q, mesh.triangles)


TINY = {
    "tetra": meshgen.regular_tetrahedron(size=0.2),
    "cube": meshgen.box(half=(0.2, 0.2, 0.2)),
    "octa": meshgen.octahedron(size=0.25),
    "ico1": meshgen.icosphere(1, radius=0.3),
    "saddle": meshgen.star_fan_solid(8, [0.06, -0.06] * 4, apex_h=0.0),
    "ruff": meshgen.star_fan_solid(6, [0.25, -0.12] * 3, apex_h=0.05, bottom=-0.25),
}


def _points_near(mesh, n, rng, spread=0.12):
    X = mesh.vertices
    tri = mesh.triangles
    t = rng.integers(0, tri.shape[0], size=n)
    bc = rng.dirichlet([1, 1, 1], size=n)
    base = np.einsum("ij,ijk->ik", bc, X[tri[t]])
    return base + rng.normal(scale=spread, size=(n, 3))


@pytest.mark.parametrize("name", sorted(TINY))
def test_distance_matches_exact_rationals(name):
    mesh = TINY[name]
    soup = mesh.soup(seed=1)
    om = oracle.OracleMesh.from_soup(soup)
    X32 = mesh.vertices.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(7)
    pts = _points_near(meshgen.Mesh(X32, mesh.triangles), 60, rng)
    d, _, _ = om.sdf_points(pts, pruned=False)
    for p, dv in zip(pts, d):
        ex = exact_ref.exact_mesh_dist2(p, X32, mesh.triangles)
        ref = math.sqrt(float(ex))
        # FP64 rounding of O(1) coordinate differences: a few ulp of 1.0, absolute
        assert abs(abs(dv) - ref) <= 8 * np.finfo(np.float64).eps, (name, p, dv, ref)


@pytest.mark.parametrize("name", sorted(TINY))
def test_sign_matches_exact_ray_parity(name):
    mesh = TINY[name]
    om = oracle.OracleMesh.from_soup(mesh.soup(seed=2))
    X32 = mesh.vertices.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(11)
    pts = _points_near(meshgen.Mesh(X32, mesh.triangles), 60, rng, spread=0.08)
    d, _, _ = om.sdf_points(pts, pruned=False)
    for p, dv in zip(pts, d):
        if abs(dv) < 1e-9:
            continue
        inside = exact_ref.exact_inside(p, X32, mesh.triangles, rng)
        assert inside is not None
        assert (dv < 0) == inside, (name, p, dv)


def test_box_closed_form():
    c, half = (0.5, 0.5, 0.5), (0.2, 0.15, 0.1)
    for sub in (1, 3):
        mesh = meshgen.box(center=c, half=half, subdiv=sub)
        om = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles)
        rng = np.random.default_rng(3 + sub)
        pts = rng.uniform(0.15, 0.85, size=(4000, 3))
        d, _, _ = om.sdf_points(pts)
        ref = exact_ref.box_sdf(pts, c, half)
        assert np.max(np.abs(d - ref)) < 1e-12


def test_tetrahedron_closed_form():
    mesh = meshgen.regular_tetrahedron(size=0.25)
    om = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles)
    V = mesh.vertices
    tri = mesh.triangles
    n = np.cross(V[tri[:, 1]] - V[tri[:, 0]], V[tri[:, 2]] - V[tri[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    off = np.einsum("ij,ij->i", n, V[tri[:, 0]])
    rng = np.random.default_rng(5)
    pts = rng.uniform(0.1, 0.9, size=(3000, 3))
    d, _, _ = om.sdf_points(pts)
    ref = np.array([exact_ref.tetra_sdf(p, V, n, off) for p in pts])
    assert np.max(np.abs(d - ref)) < 1e-12


@pytest.mark.parametrize("which", ["c1", "knot_small", "ruff"])
def test_pruned_equals_literal_loop_bitwise(which):
    if which == "c1":
        mesh = meshgen.config_mesh(1)
    elif which == "knot_small":
        mesh = meshgen.knot_tube(n_along=256, n_around=12, seed=4)
    else:
        mesh = TINY["ruff"]
    om = oracle.OracleMesh.from_soup(mesh.soup(seed=3))
    rng = np.random.default_rng(17)
    pts = np.concatenate([_points_near(mesh, 1500, rng, spread=0.03), rng.uniform(-0.2, 1.2, size=(300, 3))])
    d0, t0, r0 = om.sdf_points(pts, pruned=False)
    d1, t1, r1 = om.sdf_points(pts, pruned=True)
    assert np.array_equal(d0.view(np.int64), d1.view(np.int64))
    assert np.array_equal(t0, t1) and np.array_equal(r0, r1)
    # band queries with early exit agree with the literal loop as well
    dims, origin, h, w = (48, 48, 48), (0.0, 0.0, 0.0), 1 / 48, 3 / 48
    idx = rng.integers(0, 48 ** 3, size=3000)
    b0, bt0, _ = om.band_points(dims, origin, h, w, idx, pruned=False)
    b1, bt1, _ = om.band_points(dims, origin, h, w, idx, pruned=True)
    assert np.array_equal(b0, b1) and np.array_equal(bt0, bt1)


def test_dense_band_matches_point_queries():
    mesh = meshgen.config_mesh(1)
    om = oracle.OracleMesh.from_soup(mesh.soup(seed=1))
    dims, origin, h, w = (40, 36, 44), (0.02, -0.01, 0.0), 1 / 40, 3 / 40
    dense, tri = om.narrow_band(dims, origin, h, w, winners=True)
    idx = np.arange(np.prod(dims))
    d, t, _ = om.band_points(dims, origin, h, w, idx, pruned=False)
    assert np.array_equal(dense.ravel(), d)
    assert np.array_equal(tri.ravel(), t)
    band = np.isfinite(d)
    assert band.sum() > 1000
    assert np.all(np.abs(d[band]) < w)


def test_eikonal_in_face_regions():
    mesh = meshgen.torus(nu=40, nv=16, seed=2)
    om = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles)
    rng = np.random.default_rng(23)
    pts = _points_near(mesh, 3000, rng, spread=0.01)
    e = 1e-6
    offs = np.array([[e, 0, 0], [-e, 0, 0], [0, e, 0], [0, -e, 0], [0, 0, e], [0, 0, -e]])
    stencil = (pts[:, None, :] + np.concatenate([np.zeros((1, 3)), offs])[None]).reshape(-1, 3)
    d, t, r = om.sdf_points(stencil)
    d, t, r = d.reshape(-1, 7), t.reshape(-1, 7), r.reshape(-1, 7)
    same = np.all(t == t[:, :1], axis=1) & np.all(r == 0, axis=1) & (np.abs(d[:, 0]) > 1e-4)
    assert same.sum() > 500
    g = np.stack([(d[:, 1] - d[:, 2]), (d[:, 3] - d[:, 4]), (d[:, 5] - d[:, 6])], axis=1) / (2 * e)
    err = np.abs(np.linalg.norm(g[same], axis=1) - 1.0)
    assert err.max() < 1e-9  # d is affine in a face region: only rounding (about 3e-11 at this step) remains


def test_translation_by_grid_steps_is_an_exact_index_shift():
    mesh = _quantized(meshgen.icosphere(3, radius=0.25, displacement=0.02, seed=8))
    n, h, w = 64, 1 / 64, 3 / 64   # dyadic spacing: grid points and shifts are exact
    dims, origin = (n, n, n), (0.0, 0.0, 0.0)
    k = np.array([2, -1, 3])
    shifted = meshgen.Mesh(mesh.vertices + k * h, mesh.triangles)
    a = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles).narrow_band(dims, origin, h, w)
    b = oracle.OracleMesh.from_indexed(shifted.vertices, shifted.triangles).narrow_band(dims, origin, h, w)
    # b[z+kz, y+ky, x+kx] == a[z, y, x] wherever both are inside the grid
    sl_a = tuple(slice(max(0, -kk), n - max(0, kk)) for kk in k[::-1])
    sl_b = tuple(slice(max(0, kk), n - max(0, -kk)) for kk in k[::-1])
    assert np.array_equal(a[sl_a], b[sl_b])
    assert np.isfinite(a).sum() > 5000


def test_rotation_and_flip_permute_the_grid():
    mesh = _quantized(meshgen.icosphere(3, radius=0.25, displacement=0.03, seed=9))
    n, h, w = 32, 1 / 32, 3 / 32
    dims, origin = (n, n, n), (0.0, 0.0, 0.0)
    base = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles).narrow_band(dims, origin, h, w)
    X = mesh.vertices
    # 90 degrees about z through the domain centre: (x, y) -> (1 - y, x)   (proper rotation)
    Xr = np.stack([1.0 - X[:, 1], X[:, 0], X[:, 2]], axis=1)
    rot = oracle.OracleMesh.from_indexed(Xr, mesh.triangles).narrow_band(dims, origin, h, w)
    # new[z, j, i] at point (x_i, y_j) equals old at (y_j, 1 - x_i): old index (i_old = j, j_old = n-1-i)
    expect = np.transpose(base, (0, 2, 1))[:, :, ::-1]
    fin = np.isfinite(expect)
    assert np.array_equal(fin, np.isfinite(rot))
    assert np.max(np.abs(rot[fin] - expect[fin])) < 1e-15
    # mirror x -> 1 - x (improper: reverse triangle orientation to keep outward normals)
    Xm = np.stack([1.0 - X[:, 0], X[:, 1], X[:, 2]], axis=1)
    mir = oracle.OracleMesh.from_indexed(Xm, mesh.triangles[:, [0, 2, 1]]).narrow_band(dims, origin, h, w)
    expect = base[:, :, ::-1]
    fin = np.isfinite(expect)
    assert np.array_equal(fin, np.isfinite(mir))
    assert np.max(np.abs(mir[fin] - expect[fin])) < 1e-15


def test_random_rigid_rotation():
    mesh = meshgen.torus(nu=36, nv=14, seed=3)
    rng = np.random.default_rng(31)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    c = np.array([0.5, 0.5, 0.5])
    Xr = (mesh.vertices - c) @ q.T + c
    a = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles)
    b = oracle.OracleMesh.from_indexed(Xr, mesh.triangles)
    pts = _points_near(mesh, 3000, rng, spread=0.02)
    da, _, _ = a.sdf_points(pts)
    db, _, _ = b.sdf_points((pts - c) @ q.T + c)
    assert np.max(np.abs(da - db)) < 1e-12


@pytest.mark.parametrize("which", ["knot_small", "torus_small", "saddle", "ruff"])
def test_sign_matches_fp64_ray_parity(which):
    mesh = {"knot_small": lambda: meshgen.knot_tube(n_along=200, n_around=10, seed=6),
            "torus_small": lambda: meshgen.torus(nu=24, nv=10, seed=4),
            "saddle": lambda: TINY["saddle"], "ruff": lambda: TINY["ruff"]}[which]()
    om = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles)
    rng = np.random.default_rng(41)
    pts = _points_near(mesh, 400, rng, spread=0.02)
    d, _, _ = om.sdf_points(pts)
    keep = np.abs(d) > 1e-7
    inside = exact_ref.inside_fp64(pts[keep], mesh.vertices, mesh.triangles.astype(np.int64), seed=5)
    assert np.array_equal(d[keep] < 0, inside)


def test_sphere_sanity():
    R, f = 0.3, 6
    mesh = meshgen.icosphere(f, radius=R)
    om = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles)
    # the largest chord deviation is below R * (1 - cos(theta)), theta = longest edge angle
    X = mesh.vertices - 0.5
    tri = mesh.triangles
    cosang = np.einsum("ij,ij->i", X[tri[:, 0]], X[tri[:, 1]]) / R ** 2
    dev = R * (1 - np.cos(np.arccos(cosang.min())))
    rng = np.random.default_rng(2)
    pts = 0.5 + rng.uniform(-0.45, 0.45, size=(2000, 3))
    d, _, _ = om.sdf_points(pts)
    ref = np.linalg.norm(pts - 0.5, axis=1) - R
    assert np.max(np.abs(d - ref)) <= dev + 1e-12


def test_weld_and_classification_counts():
    for f in (2, 4):
        mesh = meshgen.icosphere(f)
        om = oracle.OracleMesh.from_soup(mesh.soup(seed=f))
        T = mesh.triangles.shape[0]
        assert om.V == T // 2 + 2 and om.E == 3 * T // 2
        assert om.n_convex == om.V and om.n_saddle == 0
        assert om.n_convex_edges == om.E
    tor = meshgen.torus(nu=30, nv=12, seed=1)
    om = oracle.OracleMesh.from_soup(tor.soup(seed=1))
    assert om.V == tor.triangles.shape[0] // 2
    assert om.n_saddle > 0  # the inner ring of a torus is hyperbolic
    cube = meshgen.box(subdiv=2)
    om = oracle.OracleMesh.from_soup(cube.soup(seed=2))
    assert om.n_flat > 0  # vertices inside the flat sides
    sad = oracle.OracleMesh.from_soup(TINY["saddle"].soup(seed=1))
    top = int(np.argmax(sad.vertices()[:, 2] * 0 + (np.abs(sad.vertices()[:, :2] - 0.5).sum(axis=1) < 1e-12)
                        * (sad.vertices()[:, 2] > 0.45)))
    assert sad.vertex_classes()[top] == 2


def test_weld_map_is_consistent():
    mesh = meshgen.config_mesh(1)
    soup = mesh.soup(seed=1)
    om = oracle.OracleMesh.from_soup(soup)
    vid = om.soup_vid()
    X = om.vertices()
    assert np.array_equal(X[vid], soup.reshape(-1, 3).astype(np.float64))


def test_invalid_meshes_are_rejected():
    mesh = meshgen.icosphere(2)
    soup = mesh.soup(seed=1)
    with pytest.raises(ValueError, match="non-manifold"):
        oracle.OracleMesh.from_soup(soup[1:])           # open surface
    flipped = soup.copy()
    flipped[0] = flipped[0][[0, 2, 1]]
    with pytest.raises(ValueError, match="non-manifold"):
        oracle.OracleMesh.from_soup(flipped)            # one flipped face
    bad = soup.copy()
    bad[3, 1, 2] = np.nan
    with pytest.raises(ValueError, match="non-finite"):
        oracle.OracleMesh.from_soup(bad)
    deg = soup.copy()
    deg[5, 2] = deg[5, 1]
    with pytest.raises(ValueError):
        oracle.OracleMesh.from_soup(deg)


def _band_loss_points(mesh, w, n, seed):
    rng = np.random.default_rng(seed)
    pts = _points_near(mesh, n, rng, spread=w / 2)
    return pts, rng.normal(size=n)


def test_adjoint_matches_finite_differences():
    mesh = meshgen.icosphere(3, radius=0.3, displacement=0.03, seed=12)
    X, tri = mesh.vertices, mesh.triangles
    w = 0.05
    pts, g = _band_loss_points(mesh, w, 4000, 3)
    om = oracle.OracleMesh.from_indexed(X, tri)
    d0, _, _ = om.sdf_points(pts)
    frozen = np.abs(d0) < w
    pts, g = pts[frozen], g[frozen]
    grad = om.adjoint_points(pts, g, w=np.inf)
    rng = np.random.default_rng(4)
    verts = rng.choice(X.shape[0], size=48, replace=False)
    eps = 1e-6
    fd, an = [], []
    for v in verts:
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, c] += eps
            Xm[v, c] -= eps
            dp, _, _ = oracle.OracleMesh.from_indexed(Xp, tri).sdf_points(pts)
            dm, _, _ = oracle.OracleMesh.from_indexed(Xm, tri).sdf_points(pts)
            fd.append(float(g @ (dp - dm)) / (2 * eps))
            an.append(grad[v, c])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= 1e-4 * np.linalg.norm(fd)


def test_adjoint_exact_identities():
    mesh = meshgen.torus(nu=40, nv=16, seed=5)
    X, tri = mesh.vertices, mesh.triangles
    om = oracle.OracleMesh.from_indexed(X, tri)
    w = 0.04
    pts, g = _band_loss_points(mesh, w, 3000, 9)
    d, _, _ = om.sdf_points(pts)
    keep = (np.abs(d) < w) & (np.abs(d) > 1e-4)
    pts, g, d = pts[keep], g[keep], d[keep]
    grad = om.adjoint_points(pts, g, w=np.inf)
    # grad_p d by central differences on the oracle
    e = 1e-7
    gp = np.zeros_like(pts)
    for c in range(3):
        off = np.zeros(3)
        off[c] = e
        dp, _, _ = om.sdf_points(pts + off)
        dm, _, _ = om.sdf_points(pts - off)
        gp[:, c] = (dp - dm) / (2 * e)
    # translation: sum_i dL/dx_i = -sum_p g_p grad_p d
    lhs = grad.sum(axis=0)
    rhs = -(g[:, None] * gp).sum(axis=0)
    assert np.allclose(lhs, rhs, rtol=1e-5, atol=1e-6 * np.abs(g).sum())
    # rotation: sum_i x_i x dL/dx_i = -sum_p p x g_p grad_p d
    lhs = np.cross(X, grad).sum(axis=0)
    rhs = -np.cross(pts, g[:, None] * gp).sum(axis=0)
    assert np.allclose(lhs, rhs, rtol=1e-5, atol=1e-6 * np.abs(g).sum())
    # homogeneity: sum_i x_i . dL/dx_i + sum_p g_p p . grad_p d = sum_p g_p d_p
    lhs = float(np.sum(X * grad) + np.sum(g * np.einsum("ij,ij->i", pts, gp)))
    assert abs(lhs - float(g @ d)) <= 1e-5 * np.abs(g).sum()


def _rotated_box_sdf(p, c, R, half):
    """Exact SDF of the box c + R diag(half) [-1, 1]^3 and the closest point of its surface."""
    q = (np.asarray(p) - c) @ R
    e = np.abs(q) - half
    d = np.linalg.norm(np.maximum(e, 0.0), axis=-1) + np.minimum(e.max(axis=-1), 0.0)
    # closest surface point from inside: push the coordinate of the nearest face out to it
    k = np.argmax(e, axis=-1)
    qs = q.copy()
    rows = np.arange(q.shape[0])
    qs[rows, k] = np.sign(q[rows, k]) * half[k]
    return d, qs @ R.T + c


@pytest.mark.parametrize("k,seed", [(2, 1), (3, 2), (4, 3)])
def test_box_union_closed_form(k, seed):
    """Union of overlapping rotated boxes (concave creases, saddle vertices where they meet box
    edges).  Outside the union, the distance to it is the smallest distance to a box.  Inside,
    -d is at least the largest depth in a box, max_j(-sdf_j), and equals it where the closest
    surface point of that box lies outside all other boxes (then it is on the union's surface).
    The sign is negative exactly inside some box."""
    mesh, boxes = meshgen.box_union(k, 600, seed=seed, return_boxes=True)
    om = oracle.OracleMesh.from_indexed(mesh.vertices, mesh.triangles)
    assert om.n_concave_edges > 0 and om.n_saddle > 0
    rng = np.random.default_rng(40 + seed)
    pts = np.concatenate([_points_near(mesh, 3000, rng, spread=0.04), rng.uniform(0.0, 1.0, size=(1000, 3))])
    d, _, _ = om.sdf_points(pts)
    sd = np.stack([_rotated_box_sdf(pts, *b)[0] for b in boxes])
    inside = (sd < -1e-12).any(axis=0)
    outside = (sd > 1e-12).all(axis=0)
    assert inside.sum() > 500 and outside.sum() > 500
    assert np.all(d[inside] < 0) and np.all(d[outside] > 0)
    assert np.max(np.abs(d[outside] - sd.min(axis=0)[outside])) < 1e-12
    depth = (-sd).max(axis=0)
    assert np.all(-d[inside] >= depth[inside] - 1e-12)
    jstar = np.argmax(-sd, axis=0)
    exact = np.zeros(pts.shape[0], dtype=bool)
    for j, b in enumerate(boxes):
        sel = inside & (jstar == j)
        _, cp = _rotated_box_sdf(pts[sel], *b)
        free = np.ones(sel.sum(), dtype=bool)
        for m2, b2 in enumerate(boxes):
            if m2 != j:
                free &= _rotated_box_sdf(cp, *b2)[0] > 1e-9
        exact[np.nonzero(sel)[0][free]] = True
    assert exact.sum() > 300
    assert np.max(np.abs(-d[exact] - depth[exact])) < 1e-12


def test_adjoint_matches_finite_differences_on_a_box_union():
    """The adjoint where the closest feature is a concave crease or a saddle vertex: a union of
    three overlapping rotated boxes, with the perturbed vertices drawn from those on the
    intersection curves (vertices inside no box face's interior grid), against central
    differences of the oracle's own distances."""
    mesh, boxes = meshgen.box_union(3, 300, seed=2, return_boxes=True)
    X, tri = mesh.vertices, mesh.triangles
    w = 0.05
    pts, g = _band_loss_points(mesh, w, 4000, 5)
    om = oracle.OracleMesh.from_indexed(X, tri)
    d0, _, _ = om.sdf_points(pts)
    frozen = np.abs(d0) < w
    pts, g = pts[frozen], g[frozen]
    grad = om.adjoint_points(pts, g, w=np.inf)
    # vertices on two box surfaces at once: the creases and their corners
    sd = np.stack([_rotated_box_sdf(X, *b)[0] for b in boxes])
    crease = np.nonzero((np.abs(sd) < 1e-9).sum(axis=0) >= 2)[0]
    assert crease.size >= 12
    rng = np.random.default_rng(6)
    verts = rng.choice(crease, size=min(24, crease.size), replace=False)
    eps = 1e-6
    fd, an = [], []
    for v in verts:
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, c] += eps
            Xm[v, c] -= eps
            dp, _, _ = oracle.OracleMesh.from_indexed(Xp, tri).sdf_points(pts)
            dm, _, _ = oracle.OracleMesh.from_indexed(Xm, tri).sdf_points(pts)
            fd.append(float(g @ (dp - dm)) / (2 * eps))
            an.append(grad[v, c])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd) > 0
    assert np.linalg.norm(fd - an) <= 1e-4 * np.linalg.norm(fd)


# ------------------------------------------------------------------ the adjoint on given features
def test_adjoint_on_given_features_equals_own_winner_adjoint_bitwise():
    """Where each point's given feature is the oracle's own winner (triangle and region label from
    the point query), the given-feature adjoint and distances are bitwise those of the searching
    adjoint and of the point query (one thread, so both sum in the same order)."""
    for mesh, w in ((meshgen.torus(nu=40, nv=16, seed=5), 0.04), (meshgen.box_union(3, 300, seed=2), 0.05)):
        X, tri = mesh.vertices, mesh.triangles
        om = oracle.OracleMesh.from_indexed(X, tri)
        pts, g = _band_loss_points(mesh, w, 3000, 21)
        d, t, r = om.sdf_points(pts)
        keep = np.abs(d) < w
        pts, g, d, t, r = pts[keep], g[keep], d[keep], t[keep], r[keep]
        labels = set(r.tolist())  # face, edge and corner winners all occur
        assert 0 in labels and labels & {1, 2, 3} and labels & {4, 5, 6}
        oracle.set_num_threads(1)
        try:
            ref = om.adjoint_points(pts, g, w=np.inf)
            got, dF = om.adjoint_features(pts, g, t, r)
        finally:
            oracle.set_num_threads(oracle.num_threads_default())
        assert np.array_equal(dF, d)
        assert np.array_equal(got, ref)


def _segment_dist_sampled(p, a, b, n=200001):
    s = np.linspace(0.0, 1.0, n)
    q = a[None, :] + s[:, None] * (b - a)[None, :]
    return np.sqrt(((q - p[None, :]) ** 2).sum(axis=1).min())


def _triangle_dist_sampled(p, a, b, c, n=400):
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    m = i + j <= n
    u, v = i[m] / n, j[m] / n
    q = a[None, :] + u[:, None] * (b - a)[None, :] + v[:, None] * (c - a)[None, :]
    return np.sqrt(((q - p[None, :]) ** 2).sum(axis=1).min())


def test_given_feature_distance_against_dense_sampling():
    """The distance to a given feature that is mostly NOT the closest one (a random nearby
    triangle and a random label: the closed triangle, one of its closed edges or a corner)
    against the minimum over a dense sample of that feature: never below it by more than
    rounding, never above it by more than the sampling step."""
    mesh = meshgen.icosphere(2, radius=0.3, displacement=0.02, seed=4)
    X, tri = mesh.vertices, mesh.triangles
    om = oracle.OracleMesh.from_indexed(X, tri)
    rng = np.random.default_rng(31)
    pts, _ = _band_loss_points(mesh, 0.08, 120, 32)
    t = rng.integers(0, tri.shape[0], size=pts.shape[0])
    r = rng.integers(0, 7, size=pts.shape[0])
    _, dF = om.adjoint_features(pts, np.zeros(pts.shape[0]), t, r)
    for p, tt, rr, d in zip(pts, t, r, dF):
        A, B, C = X[tri[tt]]
        if rr == 0:
            ref, step = _triangle_dist_sampled(p, A, B, C), 0.75 * max(np.linalg.norm(B - A), np.linalg.norm(C - A),
                                                                       np.linalg.norm(C - B)) / 400
        elif rr <= 3:
            k = rr - 1
            P0, P1 = X[tri[tt, k]], X[tri[tt, (k + 1) % 3]]
            ref, step = _segment_dist_sampled(p, P0, P1), np.linalg.norm(P1 - P0) / 200000
        else:
            ref, step = np.linalg.norm(p - X[tri[tt, rr - 4]]), 0.0
        assert abs(d) <= ref + 1e-12 and abs(d) >= ref - step - 1e-12, (rr, abs(d), ref)


def test_adjoint_on_given_features_matches_finite_differences():
    """d(sum_p g_p d_F(p)) / dX for features fixed by the caller (random triangles near the
    point and random labels, so mostly not the closest feature), against central differences
    of the same given-feature distances, on a union of rotated boxes (concave creases)."""
    mesh = meshgen.box_union(3, 300, seed=2)
    X, tri = mesh.vertices, mesh.triangles
    om = oracle.OracleMesh.from_indexed(X, tri)
    rng = np.random.default_rng(41)
    pts, g = _band_loss_points(mesh, 0.05, 1500, 42)
    # a feature of a triangle near the point: its own winner's triangle or a neighbour of it
    _, t0, _ = om.sdf_points(pts)
    nb = [[] for _ in range(tri.shape[0])]
    for a in range(tri.shape[0]):
        for v in tri[a]:
            nb[a].append(v)
    vert_tris = [[] for _ in range(X.shape[0])]
    for a in range(tri.shape[0]):
        for v in tri[a]:
            vert_tris[v].append(a)
    t = np.array([rng.choice(vert_tris[tri[a, rng.integers(0, 3)]]) for a in t0], dtype=np.int32)
    r = rng.integers(0, 7, size=pts.shape[0]).astype(np.int32)
    grad, d = om.adjoint_features(pts, g, t, r)
    keep = np.abs(d) > 1e-3  # the sign (and the derivative) is smooth away from the feature
    assert keep.mean() > 0.9
    g = np.where(keep, g, 0.0)
    grad, _ = om.adjoint_features(pts, g, t, r)
    used = np.unique(tri[t[keep]].ravel())
    verts = rng.choice(used, size=min(30, used.size), replace=False)
    eps = 1e-6
    fd, an = [], []
    for v in verts:
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, c] += eps
            Xm[v, c] -= eps
            _, dp = oracle.OracleMesh.from_indexed(Xp, tri).adjoint_features(pts, g, t, r)
            _, dm = oracle.OracleMesh.from_indexed(Xm, tri).adjoint_features(pts, g, t, r)
            fd.append(float(g @ (dp - dm)) / (2 * eps))
            an.append(grad[v, c])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd) > 0
    assert np.linalg.norm(fd - an) <= 1e-4 * np.linalg.norm(fd)
