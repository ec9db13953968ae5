"""Pins of the analytic ellipsoid target used by the shape-fitting workload (CPU only)."""
import numpy as np
import torch

import meshgen


def test_ellipsoid_sdf_on_axes_and_sphere():
    axes = (0.35, 0.25, 0.2)
    c = np.array([0.5, 0.5, 0.5])
    for i, e in enumerate(axes):
        for s in (0.25, 0.4, 0.6):
            if s <= e:
                continue
            p = c.copy()
            p[i] += s
            assert abs(meshgen.ellipsoid_sdf(p[None], axes)[0] - (s - e)) < 1e-12  # outside: the axis tip
    for s in (0.0, 0.05, 0.15):  # inside on the minor axis: the minor tip
        p = c.copy()
        p[2] += s
        assert abs(meshgen.ellipsoid_sdf(p[None], axes)[0] - (s - 0.2)) < 1e-12
    # inside on the major axis near the centre the closest point leaves the axis (x_z from the surface)
    x0 = 0.05
    xc = 0.35 ** 2 * x0 / (0.35 ** 2 - 0.2 ** 2)
    zc = 0.2 * np.sqrt(1 - (xc / 0.35) ** 2)
    want = -np.hypot(x0 - xc, zc)
    assert abs(meshgen.ellipsoid_sdf((c + [x0, 0, 0])[None], axes)[0] - want) < 1e-12
    r = 0.3
    pts = c + np.random.default_rng(0).uniform(-0.5, 0.5, size=(500, 3))
    d = meshgen.ellipsoid_sdf(pts, (r, r, r))
    assert np.max(np.abs(d - (np.linalg.norm(pts - c, axis=1) - r))) < 1e-12


def test_ellipsoid_sdf_against_dense_surface_samples():
    axes = (0.35, 0.25, 0.2)
    c = np.array([0.5, 0.5, 0.5])
    u = np.linspace(0, np.pi, 1200)
    v = np.linspace(0, 2 * np.pi, 2400, endpoint=False)
    U, V = np.meshgrid(u, v, indexing="ij")
    S = np.stack([axes[0] * np.sin(U) * np.cos(V), axes[1] * np.sin(U) * np.sin(V), axes[2] * np.cos(U)], -1)
    S = S.reshape(-1, 3) + c
    rng = np.random.default_rng(1)
    pts = c + rng.uniform(-0.45, 0.45, size=(40, 3))
    d = meshgen.ellipsoid_sdf(pts, axes)
    for p, dv in zip(pts, d):
        brute = np.min(np.linalg.norm(S - p, axis=1))
        assert abs(abs(dv) - brute) < 2e-4  # the sample spacing bounds the brute-force error
        assert abs(dv) <= brute + 1e-12      # the exact distance never exceeds a sample's


def test_ellipsoid_sdf_torch_matches_numpy():
    rng = np.random.default_rng(2)
    pts = 0.5 + rng.uniform(-0.5, 0.5, size=(2000, 3))
    a = meshgen.ellipsoid_sdf(pts)
    b = meshgen.ellipsoid_sdf_torch(torch.from_numpy(pts)).numpy()
    assert np.max(np.abs(a - b)) < 1e-12
