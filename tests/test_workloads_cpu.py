"""The seeded input generators (paper_1607_02427_gb300/workloads.py), which
feed both the oracle and the CUDA path:

* the rounded measures against Steiner's formula written out per shape;
* every named workload at its stated packing fraction, with a start in which
  no two bounding spheres are within one WCA cutoff (zero energy);
* unit orientations, zero momentum per replica, the Maxwell temperature;
* the batch's stated ranges; determinism of the seeds.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_1607_02427_gb300 import workloads as W


# ---- Steiner's formula, written out per shape --------------------------------

def _tet_wedge(a):
    # 6 edges, exterior angle pi - arccos(1/3); the mean-width term is half of
    # the sum of edge length times exterior angle
    return 6 * a * (math.pi - math.acos(1.0 / 3.0)) / 2


@pytest.mark.parametrize("a,r", [(1.0, 0.15), (4.24, 0.5)])
def test_square_area(a, r):
    assert W.outer_measure(W.square(a, r)) == pytest.approx(a * a + 4 * a * r + math.pi * r * r,
                                                            rel=1e-14)


@pytest.mark.parametrize("a,r", [(1.0, 0.15), (2.0, 0.1)])
def test_cube_volume(a, r):
    want = a ** 3 + 6 * a * a * r + 3 * math.pi * a * r * r + 4 / 3 * math.pi * r ** 3
    assert W.outer_measure(W.cube(a, r)) == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("a,r", [(1.0, 0.15), (8.49, 0.5)])
def test_tetrahedron_volume(a, r):
    want = (a ** 3 / (6 * math.sqrt(2)) + math.sqrt(3) * a * a * r + _tet_wedge(a) * r * r
            + 4 / 3 * math.pi * r ** 3)
    assert W.outer_measure(W.tetrahedron(a, r)) == pytest.approx(want, rel=1e-12)


def test_sphere_volume():
    assert W.outer_measure(W.sphere(0.5)) == pytest.approx(math.pi / 6, rel=1e-15)


def test_outer_volume_monte_carlo():
    """The octahedron's rounded volume against a point count: a point is
    inside when its distance to the solid octahedron |x|+|y|+|z| <= R is at
    most r."""
    R, r = 1.0, 0.1
    sh = W.octahedron(R, r)
    rng = np.random.default_rng(5)
    ext = R + r
    p = rng.uniform(-ext, ext, size=(400_000, 3))
    # By symmetry fold p into the positive orthant; there the solid is
    # {q >= 0, sum q <= R}, and a point outside it is nearest to the simplex
    # face sum q = R, q >= 0 (Euclidean projection by the sort-based method).
    a = np.sort(np.abs(p), axis=1)[:, ::-1]
    inside = a.sum(1) <= R
    cs = np.cumsum(a, 1)
    k = np.arange(1, 4)
    cond = a - (cs - R) / k > 0
    rho = cond.sum(1)
    theta = (cs[np.arange(len(a)), rho - 1] - R) / rho
    q = np.maximum(a - theta[:, None], 0)
    d = np.where(inside, 0.0, np.linalg.norm(a - q, axis=1))
    frac = np.mean(d <= r)
    want = W.outer_measure(sh)
    got = frac * (2 * ext) ** 3
    se = math.sqrt(frac * (1 - frac) / len(p)) * (2 * ext) ** 3
    assert abs(got - want) < 4 * se, (got, want, se)


# ---- mass properties of general polygons and polyhedra ------------------------

@pytest.mark.parametrize("mk,I", [
    (lambda: W.cube(1.0), [1 / 6] * 3),
    (lambda: W.tetrahedron(1.0), [1 / 20] * 3),
    (lambda: W.octahedron(1.0), [1 / 5] * 3),
    (lambda: W.triangular_prism(1.0, 1.0), [1 / 24 + 1 / 12, 1 / 24 + 1 / 12, 1 / 12]),
])
def test_polyhedron_mass_properties_closed_forms(mk, I):
    sh = mk()
    vol, cen, inertia = W.polyhedron_mass_properties(sh["verts"], sh["faces"])
    assert vol == pytest.approx(sh["inner_measure"], rel=1e-12)
    assert np.abs(cen).max() < 1e-12
    np.testing.assert_allclose(inertia, np.diag(I), atol=1e-12)


def test_polygon_mass_properties_closed_forms():
    for sh in (W.square(1.3), W.polygon(7, 0.9)):
        area, cen, iz = W.polygon_mass_properties(sh["verts"])
        assert area == pytest.approx(sh["inner_measure"], rel=1e-12)
        assert np.abs(cen).max() < 1e-12
        assert iz == pytest.approx(sh["inertia"][0], rel=1e-12)


def test_concave_shapes_centred():
    """The L-shape (I_z = 11 a^2 / 18, area 3 a^2) and the dented cube
    (volume a^3 - a^2 h / 3; centroid shift (a^2 h / 3)(a/2 - h/4) / V;
    I_zz = (a^5/6 - a^4 h / 30) / V) in closed form, centred."""
    a = 0.8
    L = W.l_shape2d(a, 0.1)
    area, cen, iz = W.polygon_mass_properties(L["verts"])
    assert area == pytest.approx(3 * a * a, rel=1e-12) and np.abs(cen).max() < 1e-12
    assert iz == pytest.approx(11 * a * a / 18, rel=1e-12) == L["inertia"][0]
    a, h = 1.2, 0.4
    D = W.dented_cube(a, h, 0.1)
    V = a ** 3 - a * a * h / 3
    vol, cen, inertia = W.polyhedron_mass_properties(D["verts"], D["faces"])
    assert vol == pytest.approx(V, rel=1e-12) and np.abs(cen).max() < 1e-12
    shift = (a * a * h / 3) * (a / 2 - h / 4) / V
    assert D["verts"][0, 2] == pytest.approx(-a / 2 + shift, rel=1e-12)
    assert inertia[2, 2] == pytest.approx((a ** 5 / 6 - a ** 4 * h / 30) / V, rel=1e-12)
    assert np.abs(inertia - np.diag(np.diag(inertia))).max() < 1e-12


# ---- the named workloads ----------------------------------------------------

def _phi(system, k=0):
    box = system.target_box if system.target_box is not None else system.box
    sl = system.replica_slices()[k]
    meas = sum(W.outer_measure(system.shapes[int(s)]) for s in system.shape_id[sl])
    return meas / float(np.prod(box[k][:system.dim]))


def _min_gap(system, k=0):
    """Smallest centre distance of replica k (minimum image) minus twice the
    bounding radius plus the WCA cutoff: >= 0 means no pair is in range."""
    sl = system.replica_slices()[k]
    pos = system.pos[sl]
    box = system.box[k][:system.dim]
    assert np.all(pos >= 0) and np.all(pos < box)
    tree = cKDTree(pos, boxsize=box)
    dist, _ = tree.query(pos, k=2)
    dmin = float(dist[:, 1].min())
    R = max(W.circumradius(system.shapes[int(s)]) for s in np.unique(system.shape_id[sl]))
    sh0 = system.shapes[int(system.shape_id[sl][0])]
    cut = W.wca_cut(sh0, sh0, system.sigma)
    return dmin - (2 * R + cut)


SMALL = {
    "squares": lambda: (W.config_squares_2d(), 0.50),
    "cubes": lambda: (W.config_cubes_4096(n_side=10), 0.40),
    "octahedra": lambda: (W.config_octahedra(cells=(4, 4, 8)), 0.50),
    "large": lambda: (W.config_large(counts=(8, 16, 16)), 0.55),
    "paper_cubes": lambda: (W.config_paper_table("cube", 256), 0.45),
    "paper_icosahedra": lambda: (W.config_paper_table("icosahedron", 4096), 0.45),
    "drift_squares": lambda: (W.config_energy_drift("square", 16, 0.5), 0.50),
    "drift_tetrahedra": lambda: (W.config_energy_drift("tetrahedron", 8, 0.4), 0.40),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_density_and_safe_start(name):
    s, phi = SMALL[name]()
    assert _phi(s) == pytest.approx(phi, rel=1e-12)
    assert _min_gap(s) >= -1e-9, name


@pytest.mark.parametrize("name", ["squares", "cubes", "drift_tetrahedra"])
def test_thermal_draws(name):
    s, _ = SMALL[name]()
    m = s.masses()[:, None]
    assert np.abs((m * s.vel).sum(0)).max() < 1e-9 * s.n
    # Maxwell: each velocity component ~ N(0, kT/m), kT = 1
    v2 = float(np.mean(m * s.vel ** 2))
    assert abs(v2 - 1.0) < 5 * math.sqrt(2.0 / s.vel.size)
    if s.dim == 3:
        assert np.abs(np.linalg.norm(s.orient, axis=1) - 1).max() < 1e-12
        # body-frame angular momentum components ~ N(0, I_k kT)
        from paper_1607_02427_gb300.workloads import _rotmat
        lb = np.einsum("nji,nj->ni", _rotmat(s.orient), s.angmom)
        z = lb / np.sqrt(s.inertia())
        assert abs(float(np.mean(z ** 2)) - 1.0) < 5 * math.sqrt(2.0 / z.size)


def test_batched_ranges():
    s = W.config_batched(n_replicas=24)
    assert s.n_replicas == 24
    assert np.all((s.replica_sizes >= 128) & (s.replica_sizes <= 2048))
    phis = s.params["phi"]
    for k in range(s.n_replicas):
        sl = s.replica_slices()[k]
        assert np.all(s.shape_id[sl] == k)
        sh = s.shapes[k]
        assert len(sh["verts"]) == [8, 4, 6][k % 3]
        assert 0.1 <= sh["rounding"] <= 0.2
        assert 0.30 <= phis[k] <= 0.55
        assert _phi(s, k) == pytest.approx(phis[k], rel=1e-12)
        assert _min_gap(s, k) >= -1e-9
        m = s.masses()[sl, None]
        assert np.abs((m * s.vel[sl]).sum(0)).max() < 1e-9 * s.replica_sizes[k]


def test_seeds_deterministic():
    a, b = W.config_cubes_4096(n_side=6), W.config_cubes_4096(n_side=6)
    for f in ("pos", "orient", "vel", "angmom", "box"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = W.config_cubes_4096(n_side=6, seed_index=11)
    assert not np.array_equal(a.orient, c.orient)


def test_sample_like_keeps_density():
    s = W.config_batched(n_replicas=3)
    rep = s.replica(0)
    smp = W.sample_like(s, n_target=512)
    rho_rep = rep.n / float(np.prod(rep.target_box[0]))
    rho_smp = smp.n / float(np.prod(smp.box[0]))
    assert rho_smp == pytest.approx(rho_rep, rel=1e-12)
    assert smp.n == 512
