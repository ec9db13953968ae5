"""Writes tests/golden/c1_oracle_points.txt from the FP64 oracle alone.

The 64^3 / band 3h icosphere workload (320 triangles, radius 0.3) is evaluated by
the oracle's literal triangle loop (Eq. 1 with the pseudonormal sign rule of
Section 4.3) at 400 seeded grid points near the surface.  The file is a
regression pin: a later change to the oracle's arithmetic must reproduce it, or
its commit must name the passage of the paper that justifies the change.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import meshgen  # noqa: E402
import oracle  # noqa: E402


def main():
    n, w = 64, 3 / 64
    om = oracle.OracleMesh.from_soup(meshgen.config_soup(1))
    rng = np.random.Generator(np.random.PCG64(353_101))
    idx = rng.integers(0, n ** 3, size=200_000)
    pts = oracle.grid_points((n, n, n), (0, 0, 0), 1 / n, idx)
    near = np.abs(np.linalg.norm(pts - 0.5, axis=1) - 0.3) < 1.2 * w
    idx = np.unique(idx[near])
    idx = np.sort(rng.choice(idx, size=400, replace=False))
    d, t, r = om.band_points((n, n, n), (0, 0, 0), 1 / n, w, idx, pruned=False)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_oracle_points.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle regression pin: icosphere nu=4 r=0.3, grid 64^3 on [0,1]^3, band 3h\n")
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        f.write("# linear_index  signed_distance(repr)  triangle  region\n")
        for a, b, c, e in zip(idx, d, t, r):
            f.write(f"{int(a)} {float(b)!r} {int(c)} {int(e)}\n")


if __name__ == "__main__":
    main()
