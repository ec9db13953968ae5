"""Independent references used to pin the FP64 oracle (test-side only).

* exact squared point-triangle distance in rationals (fractions.Fraction), found by
  minimising |a + s(b-a) + t(c-a) - p|^2 over the closed triangle through its 2x2
  normal equations (interior critical point) and the three clamped edge minima;
* exact ray-parity inside test in rationals (Moller-Trumbore in exact arithmetic,
  re-cast on edge or vertex hits);
* a vectorised FP64 ray-parity test with re-casting near degenerate hits, for
  larger meshes;
* closed-form signed distances of an axis-aligned box and of a regular
  tetrahedron (projection onto the simplex by enumeration of its faces).
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def _F(x) -> Fraction:
    return Fraction(float(x))


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def exact_tri_dist2(p, a, b, c) -> Fraction:
    """Exact min over the closed triangle of |x - p|^2 (all inputs converted exactly)."""
    p, a, b, c = ([_F(v) for v in x] for x in (p, a, b, c))
    e1, e2, ap = _sub(b, a), _sub(c, a), _sub(p, a)
    g11, g12, g22 = _dot(e1, e1), _dot(e1, e2), _dot(e2, e2)
    r1, r2 = _dot(ap, e1), _dot(ap, e2)
    det = g11 * g22 - g12 * g12
    cands = []
    if det != 0:
        s = (r1 * g22 - r2 * g12) / det
        t = (g11 * r2 - g12 * r1) / det
        if s >= 0 and t >= 0 and s + t <= 1:
            x = tuple(a[i] + s * e1[i] + t * e2[i] for i in range(3))
            d = _sub(x, p)
            cands.append(_dot(d, d))
    for u, v in ((a, b), (b, c), (c, a)):
        e = _sub(v, u)
        den = _dot(e, e)
        t = _dot(_sub(p, u), e) / den
        t = min(max(t, Fraction(0)), Fraction(1))
        x = tuple(u[i] + t * e[i] for i in range(3))
        d = _sub(x, p)
        cands.append(_dot(d, d))
    return min(cands)


def exact_mesh_dist2(p, X, tri) -> Fraction:
    return min(exact_tri_dist2(p, X[t[0]], X[t[1]], X[t[2]]) for t in tri)


def exact_inside(p, X, tri, rng, max_tries: int = 20):
    """Exact ray parity: True inside, False outside, None if p lies on the surface."""
    P = [_F(v) for v in p]
    Xf = [[_F(v) for v in x] for x in X]
    for _ in range(max_tries):
        r = tuple(Fraction(int(v), 1 << 20) for v in rng.integers(-(1 << 20), 1 << 20, size=3))
        if r == (0, 0, 0):
            continue
        hits, bad = 0, False
        for t in tri:
            a, b, c = Xf[t[0]], Xf[t[1]], Xf[t[2]]
            e1, e2 = _sub(b, a), _sub(c, a)
            Pv = _cross(r, e2)
            det = _dot(e1, Pv)
            Tv = _sub(P, a)
            if det == 0:
                # ray parallel to the plane; if p is in the plane the cast is ambiguous
                if _dot(Tv, _cross(e1, e2)) == 0:
                    bad = True
                    break
                continue
            u = _dot(Tv, Pv) / det
            Q = _cross(Tv, e1)
            v = _dot(r, Q) / det
            tau = _dot(e2, Q) / det
            if tau < 0 or u < 0 or v < 0 or u + v > 1:
                continue
            if tau == 0:
                return None  # on the surface
            if u == 0 or v == 0 or u + v == 1:
                bad = True  # through an edge or vertex: re-cast
                break
            hits += 1
        if not bad:
            return hits % 2 == 1
    raise RuntimeError("ray parity: no clean direction found")


def inside_fp64(pts: np.ndarray, X: np.ndarray, tri: np.ndarray, seed: int = 0, n_rays: int = 3) -> np.ndarray:
    """FP64 ray parity with re-casting when a hit is within 1e-9 of an edge; majority of n_rays."""
    rng = np.random.default_rng(seed)
    a, b, c = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    e1, e2 = b - a, c - a
    votes = np.zeros(len(pts), dtype=np.int64)
    for p_i, p in enumerate(pts):
        got = []
        tries = 0
        while len(got) < n_rays and tries < 50:
            tries += 1
            r = rng.normal(size=3)
            r /= np.linalg.norm(r)
            Pv = np.cross(r, e2)
            det = np.einsum("ij,ij->i", e1, Pv)
            Tv = p - a
            with np.errstate(divide="ignore", invalid="ignore"):
                u = np.einsum("ij,ij->i", Tv, Pv) / det
                Q = np.cross(Tv, e1)
                v = (Q @ r) / det
                tau = np.einsum("ij,ij->i", e2, Q) / det
            ok = np.abs(det) > 1e-300
            hit = ok & (tau > 0) & (u >= 0) & (v >= 0) & (u + v <= 1)
            margin = np.minimum(np.minimum(u, v), 1 - u - v)
            if np.any(hit & (margin < 1e-9)):
                continue
            got.append(int(hit.sum()) % 2)
        votes[p_i] = int(sum(got) * 2 > len(got))
    return votes.astype(bool)


def box_sdf(p: np.ndarray, center, half) -> np.ndarray:
    """Exact SDF of an axis-aligned box: |max(q,0)| + min(max_i q_i, 0), q = |p - c| - b."""
    q = np.abs(np.asarray(p) - np.asarray(center)) - np.asarray(half)
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(q.max(axis=-1), 0.0)
    return outside + inside


def simplex_projection_dist(p: np.ndarray, V: np.ndarray) -> float:
    """Distance from p to conv(V) (V: 4 points) by enumerating the simplex's faces (subsets):
    least squares on each affine hull, keeping minimisers with non-negative weights."""
    best = np.inf
    for k in range(1, 5):
        for sub in itertools.combinations(range(4), k):
            P = V[list(sub)]
            if k == 1:
                lam = np.array([1.0])
            else:
                A = (P[1:] - P[0]).T
                sol, *_ = np.linalg.lstsq(A, p - P[0], rcond=None)
                lam = np.concatenate([[1.0 - sol.sum()], sol])
            if np.all(lam >= -1e-15):
                x = lam @ P
                best = min(best, float(np.linalg.norm(p - x)))
    return best


def tetra_sdf(p: np.ndarray, V: np.ndarray, normals: np.ndarray, offsets: np.ndarray) -> float:
    """Exact SDF of a convex tetrahedron: inside -max distance to the face planes, outside the
    distance to the solid (simplex projection)."""
    s = normals @ p - offsets
    if np.all(s <= 0):
        return float(s.max())
    return simplex_projection_dist(p, V)
