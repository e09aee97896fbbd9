"""Host-side input generators (no GPU): the seeded workloads hold the
properties their recipes state."""
import math

import numpy as np

from oracle import geometry as OG
from paper_2506_20809_gb300 import inputs as I


def test_rigid_motion_keeps_shapes_gaps_and_relative_pose():
    s = I.lattice_suspension(seed=3)
    t = I.rigid_motion(s, seed=11)
    assert np.array_equal(t.kind, s.kind) and np.array_equal(t.A, s.A) and np.array_equal(t.C, s.C)
    d0 = np.linalg.norm(s.center[:, None] - s.center[None], axis=-1)
    d1 = np.linalg.norm(t.center[:, None] - t.center[None], axis=-1)
    np.testing.assert_allclose(d1, d0, atol=1e-12)
    for i, j in ((0, 1), (2, 5), (3, 7)):
        assert abs(I.separation(t, i, j) - I.separation(s, i, j)) < 1e-6
    assert not np.allclose(t.center, s.center)                    # it did move
    np.testing.assert_allclose(np.linalg.norm(t.quat, axis=1), 1.0, atol=1e-14)


def test_elongated_pair_shapes_and_gap():
    for ar in (10, 26, 64):
        for kind in (0, 1):
            s = I.elongated_pair(ar, kind, 8, gap=0.1)
            assert s.kind[0] == kind
            assert math.isclose(max(s.A[0], s.C[0]) / min(s.A[0], s.C[0]), ar, rel_tol=1e-12)
            assert math.isclose(max(s.A[0], s.C[0]), 1.0)
            g = I.separation(s, 0, 1)
            # the neighbour's centre is gap + 0.25 beyond the tip or rim; tilted,
            # it reaches closer than the gap but never touches
            assert 0.005 < g <= 0.1 + 1e-9


def test_extreme_points_lie_at_the_stated_distances():
    s = I.elongated_pair(26, 0, 8)
    d = (1e-1, 1e-2, 1e-3)
    X = I.extreme_points(s, 0, d, n_side=8)
    P = OG.SuspensionGeom.from_suspension(s).parts[0]
    dist = OG.point_spheroid_distance(P.to_local(X), s.A[0], s.C[0])
    ok = np.zeros(len(X), bool)
    for v in d:
        ok |= np.abs(dist - v) < 1e-9 * max(1.0, v) + 1e-12
    assert ok.all()


def test_serve_pool_is_reproducible_and_in_range():
    a = I.serve_pool(3, seed=5)
    b = I.serve_pool(3, seed=5)
    for s, t in zip(a, b):
        assert s.M == t.M and s.p == t.p and np.array_equal(s.center, t.center)
        assert 20 <= s.M <= 500 and s.p in (8, 12, 16)


def test_poisson_stream_rate():
    reqs = I.poisson_requests(50.0, 200.0, seed=1)
    assert abs(len(reqs) / 200.0 - 50.0) < 5.0
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] <= 200.0
    assert {r["op"] for r in reqs} == {"laplace", "stokes"}
