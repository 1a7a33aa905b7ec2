"""Host logic of bench.py's off-surface point sets: the fluid points of a workload keep the stated
clearance from every drop centre (more than the largest drop radius, so they lie outside every
drop), are seeded, and fill the drops' bounding box."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_fluid_points_keep_their_clearance_and_are_seeded():
    import bench
    from paper_1707_02156_gb300 import inputs
    w = inputs.config("c4s")
    n = 5000
    pts = bench.fluid_points(w, n, 1.6, seed=3)
    assert pts.shape == (3, n) and pts.flags["C_CONTIGUOUS"]
    cen, o = [], 0
    for p in w.p:
        k = (p + 1) ** 2
        cen.append(w.xcoef[o:o + 3 * k].reshape(3, k)[:, 0] / math.sqrt(4 * math.pi))
        o += 3 * k
    cen = np.array(cen)
    d = np.min(np.linalg.norm(pts[:, :, None] - cen.T[:, None, :], axis=0), axis=1)
    assert np.all(d > 1.6)
    assert np.all(pts >= cen.min(axis=0)[:, None]) and np.all(pts <= cen.max(axis=0)[:, None])
    assert np.array_equal(pts, bench.fluid_points(w, n, 1.6, seed=3))
    assert not np.array_equal(pts, bench.fluid_points(w, n, 1.6, seed=4))
