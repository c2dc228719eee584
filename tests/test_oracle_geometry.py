"""Pins of the oracle's nearest-point primitives against brute-force dense
sampling (Section "Model": point-line, line-line and point-plane formulae),
and of the parallel-edge rule (midpoint of overlap)."""
import numpy as np
import pytest


def _seg_samples(a, b, m):
    t = np.linspace(0.0, 1.0, m)[:, None]
    return a + t * (b - a)


def _poly_samples(poly, m):
    """Dense samples of a convex polygon (fan triangulation, barycentric grid)."""
    pts = []
    u = np.linspace(0, 1, m)
    U, V = np.meshgrid(u, u, indexing="ij")
    mask = U + V <= 1 + 1e-12
    U, V = U[mask][:, None], V[mask][:, None]
    for k in range(1, len(poly) - 1):
        a, b, c = poly[0], poly[k], poly[k + 1]
        pts.append(a + U * (b - a) + V * (c - a))
    return np.concatenate(pts, 0)


def test_point_segment_bruteforce(oracle_mod):
    rng = np.random.default_rng(1)
    m = 20001
    for _ in range(200):
        p, a, b = rng.normal(size=(3, 3))
        r, q = oracle_mod.point_segment(p, a, b)
        s = _seg_samples(a, b, m)
        dmin = np.linalg.norm(s - p, axis=1).min()
        step = np.linalg.norm(b - a) / (m - 1)
        assert r <= dmin + 1e-12 and dmin <= r + step
        assert np.linalg.norm(p - q) == pytest.approx(r, rel=1e-12, abs=1e-14)
        # q lies on the segment
        t = np.dot(q - a, b - a) / np.dot(b - a, b - a)
        assert -1e-12 <= t <= 1 + 1e-12
        assert np.linalg.norm(a + t * (b - a) - q) < 1e-12


def _random_convex_face(rng, n):
    ang = np.sort(rng.uniform(0, 2 * np.pi, n))
    rad = rng.uniform(0.5, 1.5)
    pts2 = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)  # on a circle -> convex, ccw
    # random orthonormal frame
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    c = rng.normal(size=3)
    return c + pts2 @ Q[:, :2].T, Q[:, 2]


@pytest.mark.parametrize("n", [3, 4, 5])
def test_point_face_bruteforce(oracle_mod, n):
    rng = np.random.default_rng(2 + n)
    for _ in range(60):
        poly, nrm = _random_convex_face(rng, n)
        # points both above/below and beside the face
        p = poly.mean(0) + rng.normal(size=3) * 1.2
        r, q = oracle_mod.point_face(p, poly)
        s = _poly_samples(poly, 220)
        dmin = np.linalg.norm(s - p, axis=1).min()
        assert r <= dmin + 1e-12
        assert dmin <= r + 0.02
        assert np.linalg.norm(p - q) == pytest.approx(r, rel=1e-12, abs=1e-14)
        # q lies in the face's plane
        assert abs(np.dot(q - poly[0], nrm)) < 1e-10


def test_point_face_inside_is_plane_distance(oracle_mod):
    poly = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], float)
    for z in (-0.7, 0.3, 2.0):
        r, q = oracle_mod.point_face([0.25, 0.6, z], poly)
        assert r == pytest.approx(abs(z)) and np.allclose(q, [0.25, 0.6, 0])
    # outside beyond a corner: distance to the corner
    r, q = oracle_mod.point_face([1.3, 1.4, 0.5], poly)
    assert r == pytest.approx(np.sqrt(0.09 + 0.16 + 0.25)) and np.allclose(q, [1, 1, 0])


def test_segment_segment_bruteforce(oracle_mod):
    rng = np.random.default_rng(3)
    m = 1201
    for _ in range(120):
        a1, b1, a2, b2 = rng.normal(size=(4, 3))
        r, p1, p2, par = oracle_mod.segment_segment(a1, b1, a2, b2)
        assert not par
        s1 = _seg_samples(a1, b1, m)
        s2 = _seg_samples(a2, b2, m)
        d = np.linalg.norm(s1[:, None, :] - s2[None, :, :], axis=2).min()
        step = (np.linalg.norm(b1 - a1) + np.linalg.norm(b2 - a2)) / (m - 1)
        assert r <= d + 1e-12 and d <= r + step
        assert np.linalg.norm(p1 - p2) == pytest.approx(r, rel=1e-12, abs=1e-14)


def test_segment_segment_crossing_and_skew(oracle_mod):
    # perpendicular skew segments crossing in projection: distance = offset
    r, p1, p2, _ = oracle_mod.segment_segment([-1, 0, 0], [1, 0, 0], [0, -1, 0.3], [0, 1, 0.3])
    assert r == pytest.approx(0.3) and np.allclose(p1, 0) and np.allclose(p2, [0, 0, 0.3])
    # endpoint-to-interior case
    r, p1, p2, _ = oracle_mod.segment_segment([0, 0, 0], [1, 0, 0], [2, -1, 0.5], [2, 1, 0.5])
    assert r == pytest.approx(np.hypot(1, 0.5)) and np.allclose(p1, [1, 0, 0])


def test_parallel_edge_rule_midpoint(oracle_mod):
    """Section "Model": nearly parallel edges interact at the midpoint of overlap."""
    # edge 1 on x in [0, 1]; edge 2 parallel at height 0.3 over x in [0.4, 1.8]
    r, p1, p2, par = oracle_mod.segment_segment([0, 0, 0], [1, 0, 0], [0.4, 0, 0.3], [1.8, 0, 0.3])
    assert par and r == pytest.approx(0.3)
    np.testing.assert_allclose(p1, [0.7, 0, 0], atol=1e-14)       # overlap [0.4, 1.0]
    np.testing.assert_allclose(p2, [0.7, 0, 0.3], atol=1e-14)
    # reversed direction of edge 2 gives the same overlap
    r, p1b, _, _ = oracle_mod.segment_segment([0, 0, 0], [1, 0, 0], [1.8, 0, 0.3], [0.4, 0, 0.3])
    np.testing.assert_allclose(p1b, p1, atol=1e-14)
    # nearly parallel inside the band (squared sine 1e-8 < 1e-6)
    r, p1, p2, par = oracle_mod.segment_segment([0, 0, 0], [1, 0, 0], [0.2, 1e-4, 0.3],
                                                [0.8, -1e-4, 0.3])
    assert par
    np.testing.assert_allclose(p1, [0.5, 0, 0], atol=1e-12)
    # collinear, disjoint: the closest endpoints
    r, p1, p2, par = oracle_mod.segment_segment([0, 0, 0], [1, 0, 0], [1.2, 0, 0], [2, 0, 0])
    assert par and r == pytest.approx(0.2) and np.allclose(p1, [1, 0, 0]) and np.allclose(p2, [1.2, 0, 0])
    # outside the band the rule is off: ordinary nearest points
    r, p1, p2, par = oracle_mod.segment_segment([0, 0, 0], [1, 0, 0], [0.2, 0.1, 0.3],
                                                [0.8, -0.1, 0.3])
    assert not par and np.allclose(p1, [0.5, 0, 0], atol=1e-12) and r == pytest.approx(0.3)
