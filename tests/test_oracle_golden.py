"""Regression pin of the oracle against tests/golden/c1_oracle_points.txt (written by
tests/golden/make_golden.py from the oracle alone)."""
import os

import numpy as np

import meshgen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_oracle_points.txt")


def test_oracle_reproduces_golden_points():
    rows = [ln.split() for ln in open(GOLDEN) if not ln.startswith("#")]
    idx = np.array([int(r[0]) for r in rows], dtype=np.int64)
    d_ref = np.array([float(r[1]) for r in rows])
    t_ref = np.array([int(r[2]) for r in rows])
    n, w = 64, 3 / 64
    om = oracle.OracleMesh.from_soup(meshgen.config_soup(1))
    d, t, _ = om.band_points((n, n, n), (0, 0, 0), 1 / n, w, idx, pruned=True)
    assert np.array_equal(d, d_ref)
    assert np.array_equal(t, t_ref)
    assert np.isfinite(d_ref).sum() > 200
