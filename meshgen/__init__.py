"""Seeded synthetic closed triangle meshes, emitted as FP32 triangle soups.

This module only produces inputs. It holds none of the distance-field
arithmetic: no closest-point, pseudonormal, classification or sign code lives
here, so both the CUDA path and the CPU oracle can take their inputs from it.

The meshes stand in for the paper's public STL models (Table 1: 5e4 to 2.9e6
faces of near-uniform size, Section 11.2), which are not available here. Every
mesh is built as an indexed mesh in float64, each unique vertex is rounded to
float32 once, and the soup is gathered from those rounded vertices, so copies of
a vertex in the soup are bitwise identical (the welding reading of Section 7.2).
Triangles are shuffled and each triangle's corners are rotated cyclically
(orientation preserved) so the soup carries no order (Section 7: "the order of
triangles in an STL file can be arbitrary").

Seeds follow the recipe `353_000 + config_index` (PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CENTER = np.array([0.5, 0.5, 0.5])


@dataclass
class Mesh:
    """Indexed closed mesh: float64 vertices [V,3], int32 triangles [T,3] (CCW seen from outside)."""
    vertices: np.ndarray
    triangles: np.ndarray

    def soup(self, seed: int | None = None, shuffle: bool = True) -> np.ndarray:
        """FP32 soup [T,3,3]; each unique vertex rounded once, then gathered."""
        v32 = self.vertices.astype(np.float32)
        tri = self.triangles
        if shuffle:
            rng = np.random.Generator(np.random.PCG64(0 if seed is None else seed))
            perm = rng.permutation(tri.shape[0])
            rot = rng.integers(0, 3, size=tri.shape[0])
            tri = tri[perm]
            idx = (np.arange(3)[None, :] + rot[:, None]) % 3
            tri = np.take_along_axis(tri, idx, axis=1)
        return np.ascontiguousarray(v32[tri])


# ----------------------------------------------------------------------------- helpers

def _orient_outward(vertices: np.ndarray, triangles: np.ndarray) -> np.ndarray:
    """Flip every triangle if the mesh's signed volume is negative."""
    a, b, c = (vertices[triangles[:, k]] for k in range(3))
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    if vol < 0:
        triangles = triangles[:, [0, 2, 1]]
    return np.ascontiguousarray(triangles.astype(np.int32))


def _grid_quads(nu: int, nv: int) -> np.ndarray:
    """Two triangles per quad of a doubly periodic (nu x nv) vertex grid, index = i*nv + j."""
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    i, j = i.ravel(), j.ravel()
    i1, j1 = (i + 1) % nu, (j + 1) % nv
    v00, v10, v11, v01 = i * nv + j, i1 * nv + j, i1 * nv + j1, i * nv + j1
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    return np.concatenate([t1, t2], axis=0)


# ----------------------------------------------------------------------------- icosphere

_ICO_T = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = np.array([
    (-1, _ICO_T, 0), (1, _ICO_T, 0), (-1, -_ICO_T, 0), (1, -_ICO_T, 0),
    (0, -1, _ICO_T), (0, 1, _ICO_T), (0, -1, -_ICO_T), (0, 1, -_ICO_T),
    (_ICO_T, 0, -1), (_ICO_T, 0, 1), (-_ICO_T, 0, -1), (-_ICO_T, 0, 1)], dtype=np.float64)
_ICO_F = np.array([
    (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
    (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
    (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int64)


def geodesic_directions(freq: int) -> tuple[np.ndarray, np.ndarray]:
    """Class-I geodesic subdivision of the icosahedron: unit directions [10f^2+2,3], triangles [20f^2,3].

    Each icosahedron face is split into freq^2 triangles on a barycentric lattice.
    Lattice points on shared icosahedron edges are keyed canonically so the two
    faces sharing an edge produce the same vertex index (and value).
    """
    keys: dict = {}
    pos: list = []

    def vid(a, b, c, i, j):
        # point A + (B-A) i/f + (C-A) j/f on face (a,b,c); canonical key per location
        f = freq
        k = f - i - j
        if i == f:
            key = ("v", b)
        elif j == f:
            key = ("v", c)
        elif k == f:
            key = ("v", a)
        elif k == 0:  # on edge b-c
            key = ("e",) + ((b, c, j) if b < c else (c, b, i))
        elif i == 0:  # on edge a-c
            key = ("e",) + ((a, c, j) if a < c else (c, a, k))
        elif j == 0:  # on edge a-b
            key = ("e",) + ((a, b, i) if a < b else (b, a, k))
        else:
            key = ("f", a, b, c, i, j)
        got = keys.get(key)
        if got is not None:
            return got
        if key[0] == "v":
            p = _ICO_V[key[1]]
        elif key[0] == "e":
            lo, hi, s = key[1], key[2], key[3]
            p = _ICO_V[lo] + (_ICO_V[hi] - _ICO_V[lo]) * (s / f)
        else:
            p = _ICO_V[a] + (_ICO_V[b] - _ICO_V[a]) * (i / f) + (_ICO_V[c] - _ICO_V[a]) * (j / f)
        keys[key] = len(pos)
        pos.append(p)
        return keys[key]

    tris = []
    for a, b, c in _ICO_F:
        a, b, c = int(a), int(b), int(c)
        for i in range(freq):
            for j in range(freq - i):
                p00 = vid(a, b, c, i, j)
                p10 = vid(a, b, c, i + 1, j)
                p01 = vid(a, b, c, i, j + 1)
                tris.append((p00, p10, p01))
                if i + j < freq - 1:
                    p11 = vid(a, b, c, i + 1, j + 1)
                    tris.append((p10, p11, p01))
    d = np.array(pos)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d, np.array(tris, dtype=np.int64)


def _sinusoid_field(rng, dirs: np.ndarray, n_terms: int, max_freq: float) -> np.ndarray:
    """Seeded smooth scalar field on unit directions, normalised to max |f| = 1."""
    f = np.zeros(dirs.shape[0])
    for _ in range(n_terms):
        w = rng.normal(size=3)
        w *= rng.uniform(1.0, max_freq) / np.linalg.norm(w)
        f += rng.uniform(0.5, 1.0) * np.sin(dirs @ w + rng.uniform(0, 2 * math.pi))
    return f / np.abs(f).max()


def icosphere(freq: int, radius: float = 0.3, center=CENTER, displacement: float = 0.0,
              seed: int = 0, n_terms: int = 6, max_freq: float = 3.0) -> Mesh:
    """Geodesic icosphere (20 f^2 triangles, 10 f^2 + 2 vertices), optional seeded radial displacement."""
    d, tri = geodesic_directions(freq)
    r = np.full(d.shape[0], radius)
    if displacement:
        rng = np.random.Generator(np.random.PCG64(seed))
        r = r + displacement * _sinusoid_field(rng, d, n_terms, max_freq)
    v = np.asarray(center) + d * r[:, None]
    return Mesh(v, _orient_outward(v, tri))


# ----------------------------------------------------------------------------- torus

def torus(nu: int = 250, nv: int = 100, R: float = 0.3, r: float = 0.1, bump: float = 0.02,
          jitter: float = 1e-3, seed: int = 353_001, center=CENTER) -> Mesh:
    """Torus with minor radius r + bump*sin(5u)*sin(7v) along the minor-circle normal,
    plus N(0, jitter^2) per-coordinate noise on the (welded) vertices."""
    u = 2 * math.pi * np.arange(nu) / nu
    v = 2 * math.pi * np.arange(nv) / nv
    U, Vv = np.meshgrid(u, v, indexing="ij")
    rr = r + bump * np.sin(5 * U) * np.sin(7 * Vv)
    x = (R + rr * np.cos(Vv)) * np.cos(U)
    y = (R + rr * np.cos(Vv)) * np.sin(U)
    z = rr * np.sin(Vv)
    verts = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    if jitter:
        rng = np.random.Generator(np.random.PCG64(seed))
        verts = verts + rng.normal(0.0, jitter, size=verts.shape)
    verts = verts + np.asarray(center)
    return Mesh(verts, _orient_outward(verts, _grid_quads(nu, nv)))


# ----------------------------------------------------------------------------- torus-knot tube

def knot_curve(t: np.ndarray, p: int = 3, q: int = 7, R: float = 0.3, a: float = 0.12):
    """(p,q) torus knot c(t) and its derivative, t in [0, 2pi)."""
    rho = R + a * np.cos(q * t)
    c = np.stack([rho * np.cos(p * t), rho * np.sin(p * t), a * np.sin(q * t)], axis=-1)
    drho = -a * q * np.sin(q * t)
    dc = np.stack([drho * np.cos(p * t) - rho * p * np.sin(p * t),
                   drho * np.sin(p * t) + rho * p * np.cos(p * t),
                   a * q * np.cos(q * t)], axis=-1)
    return c, dc


def _parallel_transport_frame(T: np.ndarray, P: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Closed rotation-minimising frame along a closed polyline P[n,3] with unit tangents T[n,3],
    by the double-reflection method (Wang, Juettler, Zheng and Liu, 2008): N is reflected across
    the plane normal to the chord P[i+1] - P[i], then across the plane normal to the difference
    between T[i+1] and the reflected T[i]; the closure twist is spread uniformly."""
    n = T.shape[0]
    N = np.zeros_like(T)
    a = np.cross(T[0], [0.0, 0.0, 1.0])
    if np.linalg.norm(a) < 1e-6:
        a = np.cross(T[0], [1.0, 0.0, 0.0])
    N[0] = a / np.linalg.norm(a)

    def step(Ni, Ti, Tj, chord):
        c1 = chord @ chord
        r = Ni - (2.0 / c1) * (chord @ Ni) * chord
        t = Ti - (2.0 / c1) * (chord @ Ti) * chord
        v2 = Tj - t
        c2 = v2 @ v2
        Nj = r - (2.0 / c2) * (v2 @ r) * v2 if c2 > 1e-30 else r
        Nj = Nj - (Nj @ Tj) * Tj
        return Nj / np.linalg.norm(Nj)

    for i in range(n - 1):
        N[i + 1] = step(N[i], T[i], T[i + 1], P[i + 1] - P[i])
    # transport once more from the last sample back to the first to measure the twist
    Nend = step(N[-1], T[-1], T[0], P[0] - P[-1])
    B0 = np.cross(T[0], N[0])
    phi = math.atan2(Nend @ B0, Nend @ N[0])
    ang = -phi * np.arange(n) / n
    B = np.cross(T, N)
    Nc = np.cos(ang)[:, None] * N + np.sin(ang)[:, None] * B
    Bc = np.cross(T, Nc)
    return Nc, Bc


def knot_tube(n_along: int = 8192, n_around: int = 128, radius: float = 0.04, noise: float = 0.005,
              seed: int = 353_003, p: int = 3, q: int = 7, R: float = 0.3, a: float = 0.12,
              center=CENTER) -> Mesh:
    """Closed tube around the (p,q) torus knot with seeded periodic surface noise."""
    t = 2 * math.pi * np.arange(n_along) / n_along
    c, dc = knot_curve(t, p, q, R, a)
    T = dc / np.linalg.norm(dc, axis=1, keepdims=True)
    N, B = _parallel_transport_frame(T, c)
    th = 2 * math.pi * np.arange(n_around) / n_around
    rng = np.random.Generator(np.random.PCG64(seed))
    S, TH = np.meshgrid(t, th, indexing="ij")
    field = np.zeros_like(S)
    for _ in range(8):
        fs = int(rng.integers(1, 40))
        ft = int(rng.integers(1, 9))
        field += rng.uniform(0.5, 1.0) * np.sin(fs * S + ft * TH + rng.uniform(0, 2 * math.pi))
    field /= np.abs(field).max()
    rho = radius + noise * field
    verts = (c[:, None, :] + rho[..., None] * (np.cos(TH)[..., None] * N[:, None, :]
                                               + np.sin(TH)[..., None] * B[:, None, :]))
    verts = verts.reshape(-1, 3) + np.asarray(center)
    return Mesh(verts, _orient_outward(verts, _grid_quads(n_along, n_around)))


def knot_min_strand_separation(n: int = 4096, p: int = 3, q: int = 7, R: float = 0.3, a: float = 0.12,
                               exclude: float = 0.5) -> float:
    """Smallest distance between knot-curve samples more than `exclude` apart in arc parameter."""
    t = 2 * math.pi * np.arange(n) / n
    c, _ = knot_curve(t, p, q, R, a)
    best = np.inf
    for i in range(0, n, 4):
        dt = np.abs(t - t[i])
        dt = np.minimum(dt, 2 * math.pi - dt)
        far = dt > exclude
        if far.any():
            best = min(best, float(np.linalg.norm(c[far] - c[i], axis=1).min()))
    return best


# ----------------------------------------------------------------------------- small exact shapes

def box(center=(0.5, 0.5, 0.5), half=(0.2, 0.15, 0.1), subdiv=1, axes=None) -> Mesh:
    """Box center + sum_k s_k half_k axes_k (s_k in [-1, 1]; axes: orthonormal rows, default the
    coordinate axes); each face split into quads of two triangles, subdiv segments along every
    local axis (an int, or one count per axis)."""
    c = np.asarray(center, dtype=np.float64)
    hx = np.asarray(half, dtype=np.float64)
    segs = (subdiv,) * 3 if np.isscalar(subdiv) else tuple(int(x) for x in subdiv)
    verts: dict = {}
    pos: list = []

    def vid(p):
        key = tuple(p)
        if key not in verts:
            verts[key] = len(pos)
            pos.append(p)
        return verts[key]

    tris = []
    for axis in range(3):
        for sgn in (-1, 1):
            u_ax, v_ax = [k for k in range(3) if k != axis]
            su, sv = segs[u_ax], segs[v_ax]
            for i in range(su):
                for j in range(sv):
                    quad = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = [0.0, 0.0, 0.0]
                        p[axis] = sgn
                        p[u_ax] = -1 + 2 * (i + di) / su
                        p[v_ax] = -1 + 2 * (j + dj) / sv
                        quad.append(vid(tuple(p)))
                    tris.append((quad[0], quad[1], quad[2]))
                    tris.append((quad[0], quad[2], quad[3]))
    unit = np.array(pos)
    ax = np.eye(3) if axes is None else np.asarray(axes, dtype=np.float64)
    v = c + (unit * hx) @ ax
    tri = np.array(tris, dtype=np.int64)
    # orient each triangle so its normal points away from the box centre
    a, b, cc = (v[tri[:, k]] for k in range(3))
    nrm = np.cross(b - a, cc - a)
    out = np.einsum("ij,ij->i", nrm, (a + b + cc) / 3 - c)
    tri[out < 0] = tri[out < 0][:, [0, 2, 1]]
    return Mesh(v, tri.astype(np.int32))


def dense_cluster(freq_big: int = 4, freq_small: int = 60, radius_small: float = 2e-4,
                  center_small=(0.85, 0.85, 0.85)) -> Mesh:
    """Very uneven triangle sizes in one closed mesh of two components: a coarse icosphere of large
    triangles (radius 0.3 at the domain centre) and a separate tiny, finely subdivided icosphere (a
    dense cluster: 20 freq_small^2 triangles within a few micro-units, so that tens of thousands of
    distinct vertices share a few cells of any coarse spatial hash)."""
    a = icosphere(freq_big, radius=0.3)
    b = icosphere(freq_small, radius=radius_small, center=center_small)
    v = np.concatenate([a.vertices, b.vertices])
    t = np.concatenate([a.triangles, b.triangles + a.vertices.shape[0]])
    return Mesh(v, t.astype(np.int32))


def lattice_plate(n_grid: int, half_thickness: float, offset: float, half_extent: float = 0.25,
                  subdiv: int = 24) -> Mesh:
    """A thin plate (a box) whose mid-plane is a lattice plane of the n_grid^3 cell-centre grid on
    [0, 1]^3, moved along its normal by `offset`.  The normal is (1, 2, 2)/3, so the grid points
    (i + 1/2, j + 1/2, k + 1/2)/n with i + 2j + 2k = K all lie at distance -offset from the mid-plane
    (K is chosen so that the plane passes near the domain centre), and with half_thickness = w they
    are within |offset| of the band edge, equally close to both sheets up to 2 |offset|: the
    two-sheet near tie of the FP32 winner.  Returns the mesh; the lattice index K is mesh.K."""
    nrm = np.array([1.0, 2.0, 2.0]) / 3.0
    u = np.array([2.0, 1.0, -2.0]) / 3.0
    v = np.cross(nrm, u)
    h = 1.0 / n_grid
    K = int(round((2.5 / h) - 2.5))  # n . p = h (K + 2.5) / 3 near n . (1/2, 1/2, 1/2) = 5/6
    target = h * (K + 2.5) / 3.0 + offset
    c0 = CENTER
    c = c0 + (target - float(nrm @ c0)) * nrm
    m = box(center=c, half=(half_extent, half_extent, half_thickness), subdiv=(subdiv, subdiv, 1),
            axes=np.stack([u, v, nrm]))
    m.K = K
    return m


def knife_prism(apex_deg: float = 10.0, depth: float = 0.3, length: float = 0.4, n_seg: int = 12,
                center=(0.5, 0.5, 0.5), seed: int = 0) -> Mesh:
    """A triangular prism whose cross-section has an apex angle of apex_deg (a knife edge: its two
    faces turn by 180 - apex_deg degrees), extruded over `length` in n_seg segments and rotated by
    a seeded random rotation."""
    half = depth * math.tan(math.radians(apex_deg) / 2)
    sec = np.array([[-depth / 2, 0.0], [depth / 2, half], [depth / 2, -half]])
    zs = np.linspace(-length / 2, length / 2, n_seg + 1)
    v = np.array([[x, y, z] for z in zs for x, y in sec])
    tri = []
    for s_ in range(n_seg):
        for a in range(3):
            b = (a + 1) % 3
            p0, p1, q0, q1 = 3 * s_ + a, 3 * s_ + b, 3 * (s_ + 1) + a, 3 * (s_ + 1) + b
            tri.append((p0, p1, q1))
            tri.append((p0, q1, q0))
    last = 3 * n_seg
    tri.append((0, 2, 1))
    tri.append((last, last + 1, last + 2))
    R = random_rotation(np.random.Generator(np.random.PCG64(seed)))
    v = v @ R.T + np.asarray(center)
    return Mesh(v, _orient_outward(v, np.array(tri, dtype=np.int64)))


def regular_tetrahedron(center=(0.5, 0.5, 0.5), size: float = 0.25) -> Mesh:
    """Regular tetrahedron with vertices at center + size*(+-1,+-1,+-1) (even sign parity)."""
    u = np.array([(1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)], dtype=np.float64)
    v = np.asarray(center) + size * u
    tri = np.array([(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)], dtype=np.int64)
    a, b, c = (v[tri[:, k]] for k in range(3))
    nrm = np.cross(b - a, c - a)
    out = np.einsum("ij,ij->i", nrm, (a + b + c) / 3 - np.asarray(center))
    tri[out < 0] = tri[out < 0][:, [0, 2, 1]]
    return Mesh(v, tri.astype(np.int32))


def octahedron(center=(0.5, 0.5, 0.5), size: float = 0.3) -> Mesh:
    u = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)], dtype=np.float64)
    v = np.asarray(center) + size * u
    tri = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                tri.append((sx, sy, sz))
    tri = np.array(tri, dtype=np.int64)
    a, b, c = (v[tri[:, k]] for k in range(3))
    nrm = np.cross(b - a, c - a)
    out = np.einsum("ij,ij->i", nrm, (a + b + c) / 3 - np.asarray(center))
    tri[out < 0] = tri[out < 0][:, [0, 2, 1]]
    return Mesh(v, tri.astype(np.int32))


def star_fan_solid(n: int, heights, radius: float = 0.25, apex_h: float = 0.1, bottom: float = -0.2,
                   center=(0.5, 0.5, 0.5)) -> Mesh:
    """Closed solid: a top apex joined to a ring of n rim points with per-point heights, closed by a
    bottom apex.  Alternating rim heights make the top apex a saddle; strongly folded rims give a
    ruff-like apex whose face normals point to both sides of its pseudonormal plane (Section 3.3)."""
    heights = np.asarray(heights, dtype=np.float64)
    ang = 2 * math.pi * np.arange(n) / n
    rim = np.stack([radius * np.cos(ang), radius * np.sin(ang), heights], axis=1)
    v = np.concatenate([[[0.0, 0.0, apex_h]], rim, [[0.0, 0.0, bottom]]], axis=0) + np.asarray(center)
    top, bot = 0, n + 1
    tri = []
    for i in range(n):
        a, b = 1 + i, 1 + (i + 1) % n
        tri.append((top, a, b))
        tri.append((bot, b, a))
    return Mesh(v, _orient_outward(v, np.array(tri, dtype=np.int64)))


# ----------------------------------------------------------------------------- named workloads

def config_mesh(index: int) -> Mesh:
    """The meshes of the five workloads (index 1..5; 3 is the batch, see batch_meshes)."""
    if index == 1:
        return icosphere(4, radius=0.3)
    if index == 2:
        return torus(seed=353_002)
    if index == 4:
        return knot_tube(seed=353_004)
    if index == 5:
        return icosphere(100, radius=0.3, displacement=0.02, seed=353_005)
    raise ValueError(index)


def config_soup(index: int) -> np.ndarray:
    return config_mesh(index).soup(seed=353_000 + index)


CONFIG_GRID = {1: (64, 3), 2: (512, 4), 4: (1024, 3), 5: (512, 4)}   # N, band half-width in cells


def random_rotation(rng) -> np.ndarray:
    """Uniformly distributed rotation matrix (QR of a Gaussian matrix, signs fixed, det +1)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def box_cluster(n_boxes: int, target_tris: float, seed: int, half_range=(0.06, 0.16)) -> Mesh:
    """2-4 randomly rotated boxes with pairwise disjoint bounding spheres inside [0.05, 0.95]^3,
    one closed mesh with several components; each box face is split into s x s quads so that the
    whole has about target_tris triangles.  Mostly flat edges and vertices, with sharp convex
    edges and corners: the opposite of a smooth surface for the feature classification."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = max(1, int(round(math.sqrt(target_tris / (12.0 * n_boxes)))))
    placed: list = []  # (centre, radius)
    verts, tris = [], []
    off = 0
    for _ in range(n_boxes):
        for _attempt in range(200):
            half = rng.uniform(*half_range, size=3)
            rad = float(np.linalg.norm(half))
            c = rng.uniform(0.05 + rad, 0.95 - rad, size=3) if rad < 0.45 else CENTER.copy()
            if all(np.linalg.norm(c - c2) > rad + r2 + 0.02 for c2, r2 in placed):
                break
            half_range = (half_range[0] * 0.9, half_range[1] * 0.9)
        else:
            raise RuntimeError("could not place disjoint boxes")
        placed.append((c, rad))
        b = box(center=(0.0, 0.0, 0.0), half=tuple(half), subdiv=s)
        R = random_rotation(rng)
        verts.append(b.vertices @ R.T + c)
        tris.append(b.triangles.astype(np.int64) + off)
        off += b.vertices.shape[0]
    return Mesh(np.concatenate(verts), np.concatenate(tris).astype(np.int32))


# ----------------------------------------------------------------------------- union of rotated boxes

def _rotated_box_faces(c: np.ndarray, R: np.ndarray, half: np.ndarray):
    """The 6 faces of the box c + R diag(half) [-1, 1]^3: (quad [4,3] counter-clockwise seen from
    outside, outward unit normal n, offset d) with the box on the side n.x <= d."""
    faces = []
    for k in range(3):
        u, v = R[:, (k + 1) % 3], R[:, (k + 2) % 3]
        hu, hv = half[(k + 1) % 3], half[(k + 2) % 3]
        for s in (-1.0, 1.0):
            n = s * R[:, k]
            fc = c + n * half[k]
            quad = np.array([fc - hu * u - hv * v, fc + hu * u - hv * v, fc + hu * u + hv * v, fc - hu * u + hv * v])
            if s < 0:
                quad = quad[::-1]
            faces.append((quad, n, float(n @ fc)))
    return faces


def _split_convex(poly: np.ndarray, n: np.ndarray, d: float, tol: float = 1e-12):
    """Split a planar convex polygon by the plane n.x = d: (part with n.x <= d, part with n.x >= d),
    each None when empty or degenerate; vertex order (orientation) is kept."""
    s = poly @ n - d
    if np.all(s <= tol):
        return poly, None
    if np.all(s >= -tol):
        return None, poly
    inside, outside = [], []
    m = poly.shape[0]
    for i in range(m):
        p, q = poly[i], poly[(i + 1) % m]
        sp, sq = s[i], s[(i + 1) % m]
        if sp <= tol:
            inside.append(p)
        if sp >= -tol:
            outside.append(p)
        if (sp < -tol and sq > tol) or (sp > tol and sq < -tol):
            x = p + (sp / (sp - sq)) * (q - p)
            inside.append(x)
            outside.append(x)

    def ok(pts):
        return np.array(pts) if len(pts) >= 3 else None
    return ok(inside), ok(outside)


def _weld(points: np.ndarray, tol: float) -> tuple[np.ndarray, np.ndarray]:
    """Merge points closer than tol (transitively): (unique points, index of each input point)."""
    from scipy.spatial import cKDTree
    parent = np.arange(points.shape[0])

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i
    for i, j in cKDTree(points).query_pairs(tol):
        ri, rj = find(i), find(j)
        if ri != rj:
            parent[max(ri, rj)] = min(ri, rj)
    roots = np.array([find(i) for i in range(points.shape[0])])
    uniq, idx = np.unique(roots, return_inverse=True)
    return points[uniq], idx


def _midpoint_subdivide(v: np.ndarray, t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """One level of 1-to-4 midpoint subdivision of an indexed mesh (orientation kept); an edge's
    midpoint is shared by both triangles on it."""
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    key = np.sort(e, axis=1)
    uk, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    mid = 0.5 * (v[uk[:, 0]] + v[uk[:, 1]])
    nt = t.shape[0]
    m01, m12, m20 = (v.shape[0] + inv[k * nt:(k + 1) * nt] for k in range(3))
    a, b, c = t[:, 0], t[:, 1], t[:, 2]
    out = np.concatenate([np.stack([a, m01, m20], 1), np.stack([m01, b, m12], 1),
                          np.stack([m20, m12, c], 1), np.stack([m01, m12, m20], 1)])
    return np.concatenate([v, mid]), out


def _closed_manifold(t: np.ndarray) -> bool:
    """Every directed edge occurs once and its reverse once (closed, consistently oriented, manifold)."""
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    if np.unique(e, axis=0).shape[0] != e.shape[0]:
        return False
    fwd = {tuple(x) for x in e.tolist()}
    return all((b, a) in fwd for a, b in fwd)


def _triangulate_convex(v: np.ndarray, ring: list):
    """Triangulation of a planar convex polygon (whose edges may hold extra collinear points) that
    maximises the smallest triangle quality, by the interval dynamic programme over diagonals;
    None if every triangulation has a degenerate triangle."""
    m = len(ring)
    P = v[ring]
    i, j, k = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    pa, pb, pc = P[i], P[j], P[k]
    area = 0.5 * np.linalg.norm(np.cross(pb - pa, pc - pa), axis=-1)
    e2 = ((pb - pa) ** 2).sum(-1) + ((pc - pb) ** 2).sum(-1) + ((pa - pc) ** 2).sum(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        Q = np.where(e2 > 0, 4.0 * math.sqrt(3.0) * area / e2, 0.0)
    best = np.full((m, m), np.inf)
    arg = np.zeros((m, m), dtype=np.int64)
    for span in range(2, m):
        for a in range(0, m - span):
            c = a + span
            ks = np.arange(a + 1, c)
            val = np.minimum(np.minimum(best[a, ks], best[ks, c]), Q[a, ks, c])
            t = int(np.argmax(val))
            best[a, c], arg[a, c] = val[t], ks[t]
    if best[0, m - 1] <= 1e-12:
        return None
    out, stack = [], [(0, m - 1)]
    while stack:
        a, c = stack.pop()
        if c - a < 2:
            continue
        k = int(arg[a, c])
        out.append((ring[a], ring[k], ring[c]))
        stack.extend(((a, k), (k, c)))
    return out


def _union_surface(boxes, weld_tol: float = 1e-9):
    """Boundary of the union of convex boxes as an indexed triangle mesh.

    Each face of each box is clipped against every other box: the part of a face inside box j
    is the face cut successively by j's six planes, and what is cut off on the outer side of a
    plane is kept; a face piece that ends inside j is dropped.  The kept convex pieces are
    welded; a welded vertex that lies inside an edge of a piece (a T-junction: the neighbouring
    face was cut at that point and this one was not) is inserted into that edge.  Each piece is
    then triangulated so that its worst triangle is as well shaped as possible (a fan around its
    centroid if every triangulation of it has a degenerate triangle)."""
    planes = [_rotated_box_faces(*b) for b in boxes]
    pieces = []
    for i, faces in enumerate(planes):
        for quad, _n, _d in faces:
            cells = [quad]
            for j, other in enumerate(planes):
                if j == i:
                    continue
                kept = []
                for cell in cells:
                    rest = cell
                    for _q, n, d in other:
                        rest, out = _split_convex(rest, n, d)
                        if out is not None:
                            kept.append(out)
                        if rest is None:
                            break
                    # a remaining piece lies inside box j: hidden
                cells = kept
            pieces.extend(cells)
    if not pieces:
        return None
    pts = np.concatenate(pieces)
    uv, idx = _weld(pts, weld_tol)
    polys, off = [], 0
    for p in pieces:
        ids = list(idx[off:off + p.shape[0]])
        off += p.shape[0]
        ids = [a for k, a in enumerate(ids) if a != ids[k - 1]]  # welded duplicates
        polys.append(ids)
    # T-junctions: welded vertices inside piece edges
    tris = []
    for ids in polys:
        if len(ids) < 3:
            continue
        ring = []
        for k, a in enumerate(ids):
            b = ids[(k + 1) % len(ids)]
            ring.append(a)
            pa, pb = uv[a], uv[b]
            ab = pb - pa
            rel = uv - pa
            tpar = rel @ ab / float(ab @ ab)
            off_line = np.linalg.norm(rel - tpar[:, None] * ab[None, :], axis=1)
            on = np.nonzero((off_line < 1e3 * weld_tol) & (tpar > 1e-9) & (tpar < 1 - 1e-9))[0]
            ring.extend(x for x in on[np.argsort(tpar[on])] if x != a and x != b)
        tri = _triangulate_convex(uv, ring)
        if tri is None:  # no ear with positive area left: fan around the centroid
            cidx = uv.shape[0]
            uv = np.concatenate([uv, uv[ring].mean(axis=0)[None, :]])
            tri = [(cidx, ring[k], ring[(k + 1) % len(ring)]) for k in range(len(ring))]
        tris.extend(tri)
    return uv, np.array(tris, dtype=np.int64)


def _triangle_quality(v: np.ndarray, t: np.ndarray) -> tuple[float, float]:
    """(min over triangles of 4 sqrt(3) area / sum of squared edges (1 for equilateral), min edge)."""
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    e2 = ((b - a) ** 2).sum(1) + ((c - b) ** 2).sum(1) + ((a - c) ** 2).sum(1)
    edges = np.sqrt(np.minimum(np.minimum(((b - a) ** 2).sum(1), ((c - b) ** 2).sum(1)), ((a - c) ** 2).sum(1)))
    return float((4.0 * math.sqrt(3.0) * area / e2).min()), float(edges.min())


def box_union(n_boxes: int, target_tris: float, seed: int, half_range=(0.08, 0.25),
              min_quality: float = 0.01, min_edge: float = 1e-4, return_boxes: bool = False):
    """Union of n_boxes seeded, randomly rotated, overlapping boxes as one closed mesh.

    Box j > 0 is centred at a random point inside an earlier box, so the boxes overlap and their
    union is connected.  The union's boundary is built exactly in float64 (the faces clipped
    against the other boxes, T-junctions resolved, see _union_surface) and then midpoint-
    subdivided toward target_tris triangles.  Along the intersection curves the union has
    concave edges and, where those curves meet box edges, saddle vertices.  The union is moved
    so that its bounding box is centred in the unit cube.  Placements whose triangles are too
    thin (quality below min_quality, an edge shorter than min_edge), that do not fit in
    [0.05, 0.95]^3, or that do not give a closed manifold are drawn again.  With return_boxes the boxes (centre, rotation, half-extents) come back too."""
    rng = np.random.Generator(np.random.PCG64(seed))
    for _attempt in range(2000):
        boxes = []
        for j in range(n_boxes):
            half = rng.uniform(*half_range, size=3)
            R = random_rotation(rng)
            if j == 0:
                c = CENTER + rng.uniform(-0.05, 0.05, size=3)
            else:
                cp, Rp, hp = boxes[int(rng.integers(0, j))]
                c = cp + Rp @ (rng.uniform(-0.9, 0.9, size=3) * hp)
            boxes.append((c, R, half))
        # centre the union's bounding box in the unit cube; draw again if it does not fit
        corners = np.concatenate([f[0] for b in boxes for f in _rotated_box_faces(*b)])
        lo, hi = corners.min(axis=0), corners.max(axis=0)
        if (hi - lo).max() > 0.9:
            continue
        shift = CENTER - 0.5 * (lo + hi)
        boxes = [(c + shift, R, half) for c, R, half in boxes]
        surf = _union_surface(boxes)
        if surf is None:
            continue
        v, t = surf
        if not _closed_manifold(t):
            continue
        q, emin = _triangle_quality(v, t)
        if q < min_quality or emin < min_edge:
            continue
        levels = max(0, int(round(math.log(max(target_tris, 1.0) / t.shape[0], 4))))
        for _ in range(levels):
            v, t = _midpoint_subdivide(v, t)
        mesh = Mesh(v, _orient_outward(v, t))
        return (mesh, boxes) if return_boxes else mesh
    raise RuntimeError("could not place a well-shaped box union")


def batch_meshes(n: int = 64, seed: int = 353_003, t_min: float = 1e3, t_max: float = 2e5):
    """Batch of uneven meshes: displaced icospheres, displaced tori and unions of 2-4 overlapping
    rotated boxes (type uniform), sizes log-uniform in triangles, each paired with a grid size N in
    {64, 96, ..., 384}.  Returns a list of (Mesh, N)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in range(n):
        target = math.exp(rng.uniform(math.log(t_min), math.log(t_max)))
        kind = int(rng.integers(0, 3))
        sub = 353_000 + 100 * 3 + m
        if kind == 2:
            mesh = box_union(int(rng.integers(2, 5)), target, seed=sub)
        elif kind == 0:
            f = max(2, int(round(math.sqrt(target / 20.0))))
            mesh = icosphere(f, radius=float(rng.uniform(0.2, 0.35)),
                             displacement=float(rng.uniform(0.0, 0.03)), seed=sub)
        else:
            nv = max(8, int(round(math.sqrt(target / 2.0 / 2.5))))
            nu = max(8, int(round(target / 2.0 / nv)))
            mesh = torus(nu=nu, nv=nv, R=float(rng.uniform(0.22, 0.3)), r=float(rng.uniform(0.06, 0.1)),
                         bump=float(rng.uniform(0.0, 0.02)), jitter=0.0, seed=sub)
        N = int(rng.choice(np.arange(64, 385, 32)))
        out.append((mesh, N))
    return out


# ----------------------------------------------------------------------------- analytic target field

def ellipsoid_sdf(points, axes=(0.35, 0.25, 0.2), center=CENTER, iters: int = 200):
    """Exact signed distance to an axis-aligned ellipsoid (negative inside), float64 numpy.

    For q = |p - c| (first octant by symmetry) the closest surface point is
    x_i = e_i^2 q_i / (t + e_i^2) with t the largest root of
    F(t) = sum_i (e_i q_i / (t + e_i^2))^2 - 1, monotone on (-e_m^2, inf) with e_m the
    smallest semi-axis; the root is bracketed by (-e_m^2, e_max |q|] and found by bisection
    (the monotone 1-D root find of Eberly's formulation).  When q_m = 0 and the other terms of
    F at t = -e_m^2 sum to less than 1, t = -e_m^2 and x_m follows from the surface equation."""
    p = np.asarray(points, dtype=np.float64).reshape(-1, 3) - np.asarray(center, dtype=np.float64)
    e = np.asarray(axes, dtype=np.float64)
    q = np.abs(p)
    e2 = e * e
    m = int(np.argmin(e))
    lo = np.full(q.shape[0], -e2[m])
    hi = e.max() * np.linalg.norm(q, axis=1) + 1e-300
    with np.errstate(divide="ignore", invalid="ignore"):
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            den = mid[:, None] + e2
            F = np.where(q > 0, (e * q / np.where(den > 0, den, 1.0)) ** 2, 0.0)
            F = np.where((q > 0) & (den <= 0), np.inf, F)
            pos = F.sum(axis=1) - 1.0 > 0
            lo = np.where(pos, mid, lo)
            hi = np.where(pos, hi, mid)
        t = 0.5 * (lo + hi)
        x = np.where(q > 0, e2 * q / (t[:, None] + e2), 0.0)
        # degenerate case: q_m = 0 and the root sits at t = -e_m^2
        others = [k for k in range(3) if k != m]
        xo = np.stack([e2[k] * q[:, k] / (e2[k] - e2[m]) for k in others], axis=1)
        G = sum((xo[:, j] / e[k]) ** 2 for j, k in enumerate(others))
        deg = (q[:, m] == 0) & (G < 1.0)
        if np.any(deg):
            xd = np.zeros((int(deg.sum()), 3))
            for j, k in enumerate(others):
                xd[:, k] = xo[deg, j]
            xd[:, m] = e[m] * np.sqrt(1.0 - G[deg])
            x[deg] = xd
    d = np.linalg.norm(q - x, axis=1)
    inside = ((q / e) ** 2).sum(axis=1) < 1.0
    return np.where(inside, -d, d)


def ellipsoid_sdf_torch(points, axes=(0.35, 0.25, 0.2), center=CENTER, iters: int = 100):
    """The same as ellipsoid_sdf for a torch tensor [..., 3] (float64 on its device) for points with
    no zero offset along the smallest semi-axis (always true for cell centres of an even grid
    around the centre)."""
    import torch
    p = points.to(torch.float64) - torch.tensor(center, dtype=torch.float64, device=points.device)
    e = torch.tensor(axes, dtype=torch.float64, device=points.device)
    q = p.abs()
    e2 = e * e
    lo = torch.full(q.shape[:-1], float(-e2.min()), dtype=torch.float64, device=points.device)
    hi = float(e.max()) * q.norm(dim=-1) + 1e-300
    eq = e * q
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        F = ((eq / (mid[..., None] + e2)) ** 2).sum(dim=-1) - 1.0
        pos = F > 0
        lo = torch.where(pos, mid, lo)
        hi = torch.where(pos, hi, mid)
    t = 0.5 * (lo + hi)
    x = e2 * q / (t[..., None] + e2)
    d = (q - x).norm(dim=-1)
    inside = ((q / e) ** 2).sum(dim=-1) < 1.0
    return torch.where(inside, -d, d)
