"""CPU pins of the edge-case inputs of tests/test_gpu_edge_cases.py
(Section "Model": the parallel-edge rule and the overcounting example).
They check that each construction reaches the branch it is meant to reach,
so that the GPU parity tests on them exercise those branches."""
import numpy as np
import pytest

from tests.helpers import (aligned_lattice, collinear_ridges, face_to_face, ridge_pair,
                           square_pairs_2d, swap_pair, vertex_over_face_edge)


def _ridges(s):
    """World-frame ridge segments of a ridge pair: i's top edge, j's bottom edge."""
    from tests.helpers import rotmat
    R = [rotmat(q) for q in s.orient]
    top = [p for p in (np.array([x, y, z]) for x in (-.5, .5) for y in (-.5, .5) for z in (-.5, .5))]
    zi = [R[0] @ v for v in top]
    zj = [R[1] @ v for v in top]
    hi = sorted(zi, key=lambda v: -v[2])[:2]
    lo = sorted(zj, key=lambda v: v[2])[:2]
    return [s.pos[0] + v for v in hi], [s.pos[1] + v for v in lo]


@pytest.mark.parametrize("sin2", [0.0, 1e-8, 5e-8, 1e-4])
def test_ridge_pair_squared_sine(sin2):
    """The ridges' squared sine is the one asked for (up to rounding)."""
    s = ridge_pair(sin2, 0.3, 0.28)
    (a1, b1), (a2, b2) = _ridges(s)
    d1, d2 = b1 - a1, b2 - a2
    c = np.cross(d1, d2)
    got = c @ c / ((d1 @ d1) * (d2 @ d2))
    assert got == pytest.approx(sin2, abs=1e-15)


@pytest.mark.parametrize("sin2,in_band", [(0.0, True), (1e-8, True), (5e-8, True), (1e-4, False)])
def test_ridge_pair_reaches_rule(oracle_mod, sin2, in_band):
    """In the band the parallel-edge rule moves the contact from where the
    ridges cross (x = 0.3) to the overlap's midpoint (x = 0.15): switching
    the rule off changes the torque.  Outside the band it changes nothing."""
    s = ridge_pair(sin2, 0.3, 0.28)
    on = oracle_mod.forces(s, par_eps=1e-6)
    off = oracle_mod.forces(s, par_eps=0.0)
    assert on["counts"][0, 2] > 0 and on["flags"].sum() == 0
    dt = np.abs(on["torque"] - off["torque"]).max()
    if in_band and sin2 > 0:
        assert dt > 0.05 * np.abs(off["torque"]).max()
    elif not in_band:
        assert dt == 0.0
    # exactly parallel: the ordinary solution is undefined (zero
    # determinant); the rule is the only reading
    np.testing.assert_allclose(on["force"].sum(0), 0.0, atol=1e-9 * np.abs(on["force"]).max())


def test_ridge_pair_midpoint_contact(oracle_mod):
    """Exactly parallel ridges with overlapping projections: one edge-edge
    term at the overlap's midpoint x = 0.15, at distance gap, so the
    ridge term's torque about i's centre is (0.15, 0, 0.707) x (0, 0, -f)."""
    gap = 0.28
    s = ridge_pair(0.0, 0.3, gap)
    u1, f1 = oracle_mod.wca(gap, 1.0, 0.3)
    r, p1, p2, par = oracle_mod.segment_segment([-0.5, 0, np.sqrt(0.5)], [0.5, 0, np.sqrt(0.5)],
                                                [-0.2, 0, np.sqrt(0.5) + gap],
                                                [0.8, 0, np.sqrt(0.5) + gap])
    assert par and r == pytest.approx(gap) and p1[0] == pytest.approx(0.15)


def test_no_overlap_ridges_use_endpoints(oracle_mod):
    """dx = 1.2: the projections do not overlap, and the nearest points are
    i's ridge end x = 0.5 and j's ridge start x = 0.7."""
    r, p1, p2, par = oracle_mod.segment_segment([-0.5, 0, 0], [0.5, 0, 0], [0.7, 0, 0.2],
                                                [1.7, 0, 0.2])
    assert par and r == pytest.approx(np.hypot(0.2, 0.2))
    np.testing.assert_allclose(p1, [0.5, 0, 0], atol=1e-15)
    np.testing.assert_allclose(p2, [0.7, 0, 0.2], atol=1e-15)
    s = ridge_pair(1e-8, 1.2, 0.2)
    assert oracle_mod.forces(s)["counts"][0, 2] > 0


@pytest.mark.parametrize("gap", [0.27, 0.30, 0.32, 0.335])
def test_face_to_face_terms(oracle_mod, gap):
    o = oracle_mod.forces(face_to_face(gap))
    assert o["counts"][0, 2] == 56 and o["flags"].sum() == 0


def test_collinear_ridges(oracle_mod):
    """Collinear ridges with a gap plus facing x faces: the faces give the
    56 terms of the face-to-face example (the pair is that example turned
    about x), all at the gap."""
    gap = 0.28
    o = oracle_mod.forces(collinear_ridges(gap))
    u1, _ = oracle_mod.wca(gap, 1.0, 0.3)
    assert o["counts"][0, 2] == 56
    assert o["U"][0] == pytest.approx(56 * u1, rel=1e-12)


@pytest.mark.parametrize("corner", [False, True])
def test_vertex_over_face_boundary(oracle_mod, corner):
    """The downward vertex lies exactly over the top face's edge (corner):
    its distance to i is the gap, and every term is at most r_cut away."""
    gap = 0.28
    s = vertex_over_face_edge(gap, corner)
    from tests.helpers import rotmat
    R = rotmat(s.orient[1])
    low = min((s.pos[1] + R @ np.array(v) for v in
               [(x, y, z) for x in (-.5, .5) for y in (-.5, .5) for z in (-.5, .5)]),
              key=lambda v: v[2])
    rel = low - s.pos[0]
    assert rel[1] == pytest.approx(0.5, abs=1e-14) and rel[2] == pytest.approx(0.5 + gap, abs=1e-14)
    if corner:
        assert rel[0] == pytest.approx(0.5, abs=1e-14)
    o = oracle_mod.forces(s)
    assert o["counts"][0, 2] > 0
    # the vertex-face term with i's top face is at the gap: energy >= U(gap)
    u1, _ = oracle_mod.wca(gap, 1.0, 0.3)
    assert o["U"][0] >= u1


def test_aligned_lattices(oracle_mod):
    """Aligned lattices: contacts everywhere, all at gaps in range, none
    flagged; 3D pairs are face to face, so terms come in large groups."""
    for dim, n_side in ((3, 6), (2, 12)):
        s = aligned_lattice(dim, n_side, 0.31, 0.015, dim - 1)
        o = oracle_mod.forces(s)
        assert o["counts"][0, 0] >= dim * n_side ** dim     # every lattice bond in range
        assert o["flags"].sum() == 0
        assert o["counts"][0, 2] > 4 * o["counts"][0, 0]


def test_square_pairs(oracle_mod):
    o = oracle_mod.forces(square_pairs_2d(0.3))
    assert list(o["counts"][:, 2]) == [4, 2]


def test_rule_reference_is_lower_index(oracle_mod):
    """Inside the band and not exactly parallel, the rule depends on which
    edge is the reference (the midpoint of the overlap of the other's
    projection): the oracle takes the lower-indexed particle's edge.  The
    two orders of the same ridge pair therefore differ slightly, and each
    keeps Newton's third law exactly."""
    s = ridge_pair(5e-8, 0.3, 0.28)
    a = oracle_mod.forces(s)
    b = oracle_mod.forces(swap_pair(s))
    np.testing.assert_allclose(a["force"][0], -a["force"][1], rtol=0, atol=1e-12 * 2400)
    np.testing.assert_allclose(b["force"][0], -b["force"][1], rtol=0, atol=1e-12 * 2400)
    d = np.abs(a["force"][::-1] - b["force"]).max()
    assert 1e-9 < d < 1e-3, d
    # exactly parallel: both orders agree
    s0 = ridge_pair(0.0, 0.3, 0.28)
    np.testing.assert_allclose(oracle_mod.forces(swap_pair(s0))["force"],
                               oracle_mod.forces(s0)["force"][::-1], rtol=1e-13, atol=1e-9)
