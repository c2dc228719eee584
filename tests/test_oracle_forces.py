"""Pins of the oracle's forces, torques, energies and virial (Eq. DEM,
Eq. DEM_2D, Section "Model").

* F = -grad U and tau = -dU/dtheta by central finite differences of the
  oracle's own energy (the nearest-point force is the exact gradient where
  the nearest points are unique: envelope theorem);
* Newton III and conservation of angular momentum;
* rotation and translation invariance;
* the same on clusters of concave shapes (L-shaped hexagons, dented cubes);
* the face-to-face cube and corner-to-corner square term counts (Section
  "Model", worked example; tests/golden/overcount.txt);
* zero energy when the inner shapes are separated by at least r_cut;
* the virial against finite differences of U under affine deformation.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.helpers import (SHAPES_3D, axis_angle_quat, copy_system, dent_points, nest_guests,
                           notch_points, open_cluster, quat_mul, rotmat, two_body)

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _energy(oracle_mod, s, par_eps):
    return oracle_mod.forces(s, par_eps=par_eps, scales=False)["U"].sum()


def _clusters():
    out = []
    sq = W.square(1.0, 0.15)
    out.append(("squares", open_cluster([sq], np.zeros(14, np.int32), 5)))
    out.append(("polygons", open_cluster([W.polygon(5, 0.7, 0.1), W.rod2d(1.0, 0.12), sq],
                                         np.arange(15) % 3, 6)))
    for k, (name, mk) in enumerate(SHAPES_3D.items()):
        out.append((name, open_cluster([mk()], np.zeros(10, np.int32), 20 + k)))
    out.append(("mixed3d", open_cluster([W.cube(1.0, 0.15), W.tetrahedron(1.0, 0.1),
                                         W.triangular_prism(1.0, 1.0, 0.2), W.sphere(0.3)],
                                        np.arange(12) % 4, 31)))
    # concave inner shapes (Section "Model"), with disks / spheres nested in
    # the notches / dents, within r_cut of the concave features
    L, disk = W.l_shape2d(0.6, 0.12), W.disk(0.15)
    c = open_cluster([L], np.zeros(12, np.int32), 32)
    out.append(("lshapes", nest_guests(c, range(0, 12, 2), disk, notch_points(L, 0.27), 1)))
    D, ball = W.dented_cube(1.0, 0.6, 0.12), W.sphere(0.15)
    c = open_cluster([D, W.cube(0.9, 0.1)], (np.arange(10) % 4 == 3).astype(np.int32), 33)
    out.append(("dented", nest_guests(c, [0, 1, 2, 4, 5], ball, dent_points(D, 0.27), 2)))
    return out


CLUSTERS = _clusters()


@pytest.mark.parametrize("name,s", CLUSTERS, ids=[c[0] for c in CLUSTERS])
def test_force_is_minus_gradient(oracle_mod, name, s):
    par_eps = 0.0           # parallel rule off: the potential is then conservative
    o = oracle_mod.forces(s, par_eps=par_eps)
    assert o["counts"][0, 2] > 0, "cluster must have contacts"
    h = 1e-6
    dim = s.dim
    for i in range(min(s.n, 8)):
        for a in range(dim):
            sp, sm = copy_system(s), copy_system(s)
            sp.pos[i, a] += h
            sm.pos[i, a] -= h
            fd = -(_energy(oracle_mod, sp, par_eps) - _energy(oracle_mod, sm, par_eps)) / (2 * h)
            assert fd == pytest.approx(o["force"][i, a], abs=1e-6 * (1 + o["fscale"][i]))
        axes = np.eye(3) if dim == 3 else [None]
        for k, ax in enumerate(axes):
            sp, sm = copy_system(s), copy_system(s)
            if dim == 3:
                sp.orient[i] = quat_mul(axis_angle_quat(ax, h), s.orient[i])
                sm.orient[i] = quat_mul(axis_angle_quat(ax, -h), s.orient[i])
            else:
                sp.orient[i, 0] += h
                sm.orient[i, 0] -= h
            fd = -(_energy(oracle_mod, sp, par_eps) - _energy(oracle_mod, sm, par_eps)) / (2 * h)
            assert fd == pytest.approx(o["torque"][i, k], abs=1e-6 * (1 + o["tscale"][i]))


@pytest.mark.parametrize("name,s", CLUSTERS, ids=[c[0] for c in CLUSTERS])
def test_newton3_and_angular_momentum(oracle_mod, name, s):
    o = oracle_mod.forces(s)
    F, T = o["force"], o["torque"]
    scale = o["fscale"].sum()
    assert np.abs(F.sum(0)).max() < 1e-12 * scale
    if s.dim == 3:
        L = T.sum(0) + np.cross(s.pos, F).sum(0)
    else:
        L = T[:, 0].sum() + (s.pos[:, 0] * F[:, 1] - s.pos[:, 1] * F[:, 0]).sum()
    assert np.abs(L).max() < 1e-11 * (o["tscale"].sum() + scale * np.abs(s.pos).max())


@pytest.mark.parametrize("name,s", [c for c in CLUSTERS if c[1].dim == 3],
                         ids=[c[0] for c in CLUSTERS if c[1].dim == 3])
def test_rotation_translation_invariance(oracle_mod, name, s):
    o = oracle_mod.forces(s)
    q = axis_angle_quat([0.3, -0.5, 0.8], 1.1)
    R = rotmat(q)
    c = s.box[0] / 2
    t = copy_system(s)
    t.pos = (s.pos - c) @ R.T + c + np.array([0.37, -1.2, 2.5])
    t.orient = np.array([quat_mul(q, qi) for qi in s.orient])
    o2 = oracle_mod.forces(t)
    assert o2["U"][0] == pytest.approx(o["U"][0], rel=1e-12)
    np.testing.assert_allclose(o2["force"], o["force"] @ R.T, atol=1e-9 * (1 + o["fscale"].max()))
    np.testing.assert_allclose(o2["torque"], o["torque"] @ R.T, atol=1e-9 * (1 + o["tscale"].max()))


@pytest.mark.parametrize("name,s", [c for c in CLUSTERS if c[1].dim == 2],
                         ids=[c[0] for c in CLUSTERS if c[1].dim == 2])
def test_rotation_invariance_2d(oracle_mod, name, s):
    o = oracle_mod.forces(s)
    th = 0.83
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    c = s.box[0] / 2
    t = copy_system(s)
    t.pos = (s.pos - c) @ R.T + c
    t.orient = s.orient + th
    o2 = oracle_mod.forces(t)
    # rotating centres ~200 from the origin rounds them at ~3e-14; steep
    # contacts turn that into ~1e-12 of U
    assert o2["U"][0] == pytest.approx(o["U"][0], rel=1e-11)
    np.testing.assert_allclose(o2["force"], o["force"] @ R.T, atol=1e-9 * (1 + o["fscale"].max()))
    np.testing.assert_allclose(o2["torque"], o["torque"], atol=1e-9 * (1 + o["tscale"].max()))


def _golden(name):
    vals = {}
    with open(f"{GOLDEN}/{name}") as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


@pytest.mark.parametrize("gap", [0.27, 0.30, 0.32, 0.335])
def test_face_to_face_cubes_count(oracle_mod, gap):
    """Section "Model": two cubes face to face; every interacting feature pair
    sits at the face gap.  The count is fixed in tests/golden/overcount.txt."""
    g = _golden("overcount.txt")
    s = two_body(W.cube(1.0, 0.15), W.cube(1.0, 0.15), [0, 0, 1.0 + gap], sigma=0.3)
    o = oracle_mod.forces(s)
    u1, f1 = oracle_mod.wca(gap, 1.0, 0.3)
    assert o["U"][0] == pytest.approx(g["cube_face_face_terms"] * u1, rel=1e-12)
    assert o["counts"][0, 2] == g["cube_face_face_terms"]
    assert o["counts"][0, 1] == g["cube_pair_feature_pairs"]
    np.testing.assert_allclose(o["force"][1], [0, 0, g["cube_face_face_terms"] * f1], rtol=1e-12,
                               atol=1e-9)
    assert np.abs(o["torque"]).max() < 1e-9
    # virial: x_ij (x) f_ij with x_ij = (0, 0, -(1 + gap)), f on particle 0 = (0, 0, -F)
    assert o["virial"][0, 2, 2] == pytest.approx((1 + gap) * g["cube_face_face_terms"] * f1,
                                                 rel=1e-12)


def test_overcount_isosurface_shift(oracle_mod):
    """Section "Model", worked example: the 1 kT isosurface of the face-to-
    face cube interaction lies farther out than a single term's by about 10%
    of sigma (tests/golden/overcount.txt).  The oracle's energy of two
    aligned cubes is bisected for the gap where it equals kT = epsilon; the
    single term's 1 kT gap is sigma (U(sigma) = epsilon)."""
    g = _golden("overcount.txt")
    sig = 0.3
    rc = 2 ** (1 / 6) * sig

    def U(gap):
        s = two_body(W.cube(1.0, 0.15), W.cube(1.0, 0.15), [0, 0, 1.0 + gap], sigma=sig)
        return oracle_mod.forces(s)["U"][0]

    lo, hi = sig, rc                    # U(lo) = 56 kT > kT > U(hi) = 0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if U(mid) > 1.0:
            lo = mid
        else:
            hi = mid
    shift = (0.5 * (lo + hi) - sig) / sig
    assert shift == pytest.approx(g["isosurface_shift_over_sigma"], abs=0.005)
    # the 56 terms at the gap: 56 U(gap) = kT there
    u1, _ = oracle_mod.wca(0.5 * (lo + hi), 1.0, sig)
    assert 56 * u1 == pytest.approx(1.0, rel=1e-9)


def test_squares_corner_and_edge_counts(oracle_mod):
    g = _golden("overcount.txt")
    sq = W.square(1.0, 0.15)
    gap = 0.31
    u1, _ = oracle_mod.wca(gap, 1.0, 0.3)
    s = two_body(sq, sq, [1 + gap / np.sqrt(2), 1 + gap / np.sqrt(2)], sigma=0.3)
    assert oracle_mod.forces(s)["U"][0] == pytest.approx(g["square_corner_corner_terms"] * u1,
                                                          rel=1e-12)
    s = two_body(sq, sq, [0, 1 + gap], sigma=0.3)
    assert oracle_mod.forces(s)["U"][0] == pytest.approx(g["square_edge_edge_terms"] * u1,
                                                          rel=1e-12)


def test_overcount_bound_range(oracle_mod):
    """Section "Model": overcounting never extends the interaction range
    beyond r_cut: inner shapes separated by >= r_cut do not interact."""
    rng = np.random.default_rng(9)
    shapes = list(SHAPES_3D.values())
    for trial in range(60):
        a, b = shapes[trial % 4](), shapes[(trial // 4) % 4]()
        qa, qb = W.random_quaternions(rng, 2)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        rc = W.wca_cut(a, b)
        sa = W._support(a, qa, u)
        sb = W._support(b, qb, -u)
        for extra, expect_zero in ((rc * 1.0001, True),):
            s = two_body(a, b, (sa + sb + extra) * u, qa=qa, qb=qb)
            o = oracle_mod.forces(s)
            assert o["U"][0] == 0.0 and np.all(o["force"] == 0.0)


def test_energy_positive_inside_range(oracle_mod):
    """Touching along a face normal at gap < r_cut always interacts."""
    for name, mk in SHAPES_3D.items():
        sh = mk()
        v = sh["verts"]
        f = sh["faces"][0]
        n = np.cross(v[f[1]] - v[f[0]], v[f[2]] - v[f[0]])
        n /= np.linalg.norm(n)
        h = np.dot(v[f[0]], n)
        rc = W.wca_cut(sh, sh)
        # mirror image across the face plane, at face gap 0.9 r_cut
        d = n * (2 * h + 0.9 * rc)
        s = two_body(sh, sh, d, qa=[1, 0, 0, 0], qb=[0, n[0], n[1], n[2]])
        assert oracle_mod.forces(s)["U"][0] > 0.0, name


@pytest.mark.parametrize("name,s", [c for c in CLUSTERS if c[0] in ("cube", "mixed3d", "squares")],
                         ids=["cube", "mixed3d", "squares"])
def test_virial_affine_derivative(oracle_mod, name, s):
    """dU/d(gamma) under x -> (1 + gamma E) x of the centres gives -W."""
    o = oracle_mod.forces(s, par_eps=0.0)
    W9 = o["virial"][0]
    dim = s.dim
    c = s.box[0] / 2
    h = 1e-6
    for a in range(dim):
        for b in range(dim):
            E = np.zeros((dim, dim))
            E[a, b] = 1.0
            sp, sm = copy_system(s), copy_system(s)
            sp.pos = c + (s.pos - c) @ (np.eye(dim) + h * E).T
            sm.pos = c + (s.pos - c) @ (np.eye(dim) - h * E).T
            dU = (_energy(oracle_mod, sp, 0.0) - _energy(oracle_mod, sm, 0.0)) / (2 * h)
            # x_a -> x_a + gamma x_b : dU/dgamma = sum (dU/dd)_a d_b = -W[b][a]
            assert dU == pytest.approx(-W9[b, a], abs=1e-6 * (1 + o["fscale"].sum()))


@pytest.mark.parametrize("vertex,valence", [(0, 5), (12, 6)])
def test_icosphere_vertex_valence(oracle_mod, vertex, valence):
    """A small sphere straight out from a vertex of the 80-face icosphere,
    at distance d: the vertex's nearest point on each of its incident faces
    is the vertex itself, and every other face lies beyond r_cut, so
    U = valence U(d): 5 faces meet at the icosahedron's own vertices, 6 at
    the edge midpoints the subdivision added (Eq. DEM, vertex-face terms)."""
    ico = W.icosphere(0.7, 0.02)
    tip = ico["verts"][vertex]
    d = 0.036
    s = two_body(ico, W.sphere(0.02), tip * (1 + d / np.linalg.norm(tip)), sigma=0.04)
    o = oracle_mod.forces(s)
    u1, f1 = oracle_mod.wca(d, 1.0, 0.04)
    assert o["counts"][0, 2] == valence
    assert o["U"][0] == pytest.approx(valence * u1, rel=1e-12)
    # the net force points along the vertex's radius
    np.testing.assert_allclose(o["force"][1], valence * f1 * tip / np.linalg.norm(tip), rtol=1e-9,
                               atol=1e-12 * valence * abs(f1))
