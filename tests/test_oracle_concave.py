"""Pins of the oracle on concave inner shapes (Section "Model": the inner
shape may be concave; Eq. DEM and Eq. DEM_2D sum over the same feature
pairs whatever the shape's convexity).

* A disk in the notch of the L-shaped hexagon, at distances u and v from the
  two edges that meet at the reflex vertex: exactly two terms, U = U(u) +
  U(v), and the force on the disk is (f(u), f(v)).
* A sphere on the axis of the dented cube, above the apex of the dent: the
  four dent faces are at the same distance d = t (z - z_apex) / sqrt(h^2 +
  t^2) (t the half edge, h the dent depth), so U = 4 U(d) and the force is
  4 f(d) t / sqrt(h^2 + t^2) along the axis, whatever the dented cube's
  orientation.
* A concave shape is not its convex hull: with the sphere inside the dent,
  no point of the hull's top face is within r_cut of the sphere's centre in
  the cases below, yet the energy is positive.
* Overcounting never reaches beyond r_cut of the inner shape (Section
  "Model") for concave shapes either.
"""
import math

import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.helpers import axis_angle_quat, rotmat, two_body

RC = 2.0 ** (1.0 / 6.0)


def _wca(r, sigma, eps=1.0):
    """Closed form of the shifted WCA energy and the magnitude -dU/dr."""
    if r >= RC * sigma:
        return 0.0, 0.0
    x6 = (sigma / r) ** 6
    return 4 * eps * (x6 * x6 - x6) + eps, 24 * eps * (2 * x6 * x6 - x6) / r


@pytest.mark.parametrize("u,v", [(0.20, 0.25), (0.31, 0.12), (0.15, 0.33)])
def test_disk_in_l_notch(oracle_mod, u, v):
    L = W.l_shape2d(1.0, 0.15)
    disk = W.disk(0.15)
    sigma = 0.3                      # rounding_L + rounding_disk
    corner = L["verts"][L["reflex_vertex"]]
    s = two_body(L, disk, corner + np.array([u, v]))
    o = oracle_mod.forces(s)
    uu, fu = _wca(u, sigma)
    uv, fv = _wca(v, sigma)
    assert o["U"][0] == pytest.approx(uu + uv, rel=1e-12)
    assert o["counts"][0, 2] == (u < RC * sigma) + (v < RC * sigma)
    # absolute slack: one edge's force leaks ~1e-16 of itself into the other axis
    tol = 1e-13 * (fu + fv)
    np.testing.assert_allclose(o["force"][1], [fu, fv], rtol=1e-12, atol=tol)
    np.testing.assert_allclose(o["force"][0], [-fu, -fv], rtol=1e-12, atol=tol)


@pytest.mark.parametrize("dz", [0.08, 0.12, 0.18])
@pytest.mark.parametrize("turn", [0.0, 0.7])
def test_sphere_in_dent(oracle_mod, dz, turn):
    a, depth = 1.0, 0.5
    D = W.dented_cube(a, depth, 0.1)
    ball = W.sphere(0.1)
    sigma = 0.2
    t = a / 2
    apex = D["verts"][D["apex"]]
    p_body = apex + np.array([0.0, 0.0, dz])
    q = axis_angle_quat([0.4, -0.2, 0.9], turn)
    R = rotmat(q)
    s = two_body(D, ball, R @ p_body, qa=q)
    o = oracle_mod.forces(s)
    d = t * dz / math.hypot(depth, t)
    u1, f1 = _wca(d, sigma)
    assert d < RC * sigma
    assert o["counts"][0, 2] == 4
    assert o["U"][0] == pytest.approx(4 * u1, rel=1e-12)
    f_axis = 4 * f1 * t / math.hypot(depth, t)
    np.testing.assert_allclose(o["force"][1], R @ [0, 0, f_axis], rtol=1e-11, atol=1e-13 * f_axis)
    # the hull's top face (z = top) is farther than r_cut from the sphere
    top = D["verts"][4, 2]
    assert top - p_body[2] > RC * sigma


def test_concave_range_bound(oracle_mod):
    """Inner shapes separated along some axis by at least r_cut never
    interact (the bound holds for the convex hull, hence for the shape)."""
    rng = np.random.default_rng(12)
    shapes3 = [W.dented_cube(1.0, 0.5, 0.12), W.dented_cube(1.0, 0.8, 0.1), W.cube(1.0, 0.15)]
    for trial in range(40):
        a, b = shapes3[trial % 3], shapes3[(trial // 3) % 2]
        qa, qb = W.random_quaternions(rng, 2)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        gap = W.wca_cut(a, b) * 1.0001
        s = two_body(a, b, (W._support(a, qa, u) + W._support(b, qb, -u) + gap) * u, qa=qa, qb=qb)
        o = oracle_mod.forces(s)
        assert o["U"][0] == 0.0 and np.all(o["force"] == 0.0)
    L = W.l_shape2d(1.0, 0.15)
    for trial in range(40):
        th = rng.uniform(-np.pi, np.pi, size=2)
        ang = rng.uniform(0, 2 * np.pi)
        u = np.array([np.cos(ang), np.sin(ang)])
        ha = W._support(L, np.array([th[0]]), u)
        hb = W._support(L, np.array([th[1]]), -u)
        s = two_body(L, L, (ha + hb + W.wca_cut(L, L) * 1.0001) * u, qa=th[0], qb=th[1])
        o = oracle_mod.forces(s)
        assert o["U"][0] == 0.0 and np.all(o["force"] == 0.0)
