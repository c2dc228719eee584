"""GPU parity of the pair-feature kernels (Eq. DEM, Eq. DEM_2D) against the
FP64 oracle, element by element, through the C ABI.

Inputs: seeded contact-rich random clusters in periodic boxes (2D squares,
mixed polygons / rods / disks, 3D cubes, tetrahedra, octahedra, prisms,
spheres and mixtures, and the concave L-shaped hexagon and dented cube), sizes that span several thread blocks with a ragged
tail, multi-replica batches mixing cell-list and all-pairs replicas, and
edge cases (a lone particle, particles with no contacts, a tiny neighbour
list that must grow).  Tolerances and error measures: tests/gpu_common.py.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import TOL, assert_parity, compare_forces, force_errors, load_dem
from tests.helpers import dent_points, nest_guests, notch_points

pytestmark = pytest.mark.gpu

PRECISIONS = [0, 1, 2]
PNAMES = {0: "fp64", 1: "fp32", 2: "fp32c"}


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _periodic_cluster(shapes, ids, box, seed, **kw):
    rng = np.random.default_rng(seed)
    return W.contact_cluster(shapes, np.asarray(ids, np.int32), box, rng, **kw)


def _systems():
    out = {}
    out["squares"] = lambda: _periodic_cluster([W.square(1.0, 0.15)], np.zeros(200, int),
                                               [30.0, 30.0], 1, sigma=0.3)
    out["polys2d"] = lambda: _periodic_cluster(
        [W.polygon(5, 0.7, 0.1), W.rod2d(1.0, 0.12), W.square(1.0, 0.15), W.disk(0.2, 0.02)],
        np.arange(200) % 4, [30.0, 30.0], 2)
    out["disks"] = lambda: _periodic_cluster([W.disk(0.25)], np.zeros(400, int), [25.0, 25.0], 3)
    # 32 vertices and 32 edges: every bit of the feature masks in use
    out["poly32"] = lambda: _periodic_cluster([W.polygon(32, 0.8, 0.1)], np.zeros(200, int),
                                              [40.0, 40.0], 11)
    out["cubes"] = lambda: _periodic_cluster([W.cube(1.0, 0.15)], np.zeros(333, int),
                                             [14.0, 14.0, 14.0], 4, sigma=0.3)
    out["tets"] = lambda: _periodic_cluster([W.tetrahedron(1.0, 0.15)], np.zeros(300, int),
                                            [11.0, 11.0, 11.0], 5)
    out["octas"] = lambda: _periodic_cluster([W.octahedron(1.0, 0.1)], np.zeros(300, int),
                                             [15.0, 15.0, 15.0], 6)
    out["prisms"] = lambda: _periodic_cluster([W.triangular_prism(1.0, 1.0, 0.2)],
                                              np.zeros(300, int), [12.0, 12.0, 12.0], 7)
    out["spheres"] = lambda: _periodic_cluster([W.sphere(0.3, 0.036)], np.zeros(400, int),
                                               [9.0, 9.0, 9.0], 8)
    out["icosas"] = lambda: _periodic_cluster([W.icosahedron(0.8, 0.15)], np.zeros(250, int),
                                              [12.0, 12.0, 12.0], 10)
    # concave inner shapes (Section "Model"): the L-shaped hexagon with disks,
    # the dented cube with cubes and spheres
    # (disks / spheres nested in the notches / dents, within r_cut of the
    # concave features)
    L, D = W.l_shape2d(0.6, 0.12), W.dented_cube(1.0, 0.6, 0.12)
    out["lshapes"] = lambda: nest_guests(
        _periodic_cluster([L], np.zeros(180, int), [30.0, 30.0], 12),
        range(0, 180, 2), W.disk(0.15, 0.01), notch_points(L, 0.27), 12)
    out["dented"] = lambda: nest_guests(
        _periodic_cluster([D, W.cube(0.9, 0.1)], np.arange(220) % 2, [14.0, 14.0, 14.0], 13),
        range(0, 220, 2), W.sphere(0.15, 0.009), dent_points(D, 0.27), 13)
    out["mixed3d"] = lambda: _periodic_cluster(
        [W.cube(1.0, 0.15), W.tetrahedron(1.0, 0.1), W.triangular_prism(1.0, 1.0, 0.2),
         W.sphere(0.3, 0.036), W.octahedron(0.9, 0.12)], np.arange(290) % 5,
        [13.0, 13.0, 13.0], 9)
    return out


SYSTEMS = _systems()
_cache = {}


def system(name):
    if name not in _cache:
        _cache[name] = SYSTEMS[name]()
    return _cache[name]


DECOMPS = {"thread": 1, "warp": 2, "staged": 3, "split": 4}


@pytest.mark.parametrize("decomp", list(DECOMPS))
@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_forces_parity(dem, name, precision, decomp):
    s = system(name)
    errs, ref, _ = compare_forces(dem, s, precision, decomp=DECOMPS[decomp])
    assert ref["counts"][0, 2] > 0, "input must have contacts"
    assert_parity(errs, precision, f"{name}/{PNAMES[precision]}/{decomp}")


@pytest.mark.parametrize("name", ["cubes", "mixed3d", "polys2d"])
def test_decompositions_same_work(dem, name):
    """All decompositions run the same culls on the same items: every work
    counter agrees exactly (FP64 mode, so no test sits at a rounding edge).
    Vertex transforms [3] are left out: STAGED maps a vertex only when the
    other shape has a masked face (or 2D edge) for it."""
    s = system(name)
    keep = [k for k in range(18) if k not in (3, 13, 14)]
    cnt = {}
    for nm, dec in DECOMPS.items():
        with dem.DEM(s, dem.DEM_FP64, decomp=dec) as d:
            cnt[nm] = d.counters()[keep]
    for nm in DECOMPS:
        np.testing.assert_array_equal(cnt[nm], cnt["thread"], err_msg=nm)


def test_autotune_keeps_results(dem):
    s = system("cubes")
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        f0, _ = d.forces()
        dem.dem_autotune(d.ctx)
        assert d.get_param("decomp") in (1.0, 2.0, 3.0, 4.0)
        assert d.get_param("autotune_ms_4") > 0
        f1, _ = d.forces()
        d.step(5, 1e-3, dem.DEM_NVE)
    scale = np.abs(f0).max()
    assert np.abs(f1 - f0).max() <= 1e-5 * scale


@pytest.mark.parametrize("decomp", list(DECOMPS))
@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
def test_batched_replicas(dem, precision, decomp):
    """Replicas of different shapes and sizes in one launch, including
    replicas small enough for the all-pairs search and a one-particle one."""
    reps = [system("cubes"), system("tets").replica(0),
            _periodic_cluster([W.triangular_prism(1.0, 1.0, 0.15)], np.zeros(24, int),
                              [5.5, 5.5, 5.5], 21, gap=(0.9, 1.2), gap_min=0.85),
            _periodic_cluster([W.cube(1.0, 0.12)], np.zeros(1, int), [6.0, 6.0, 6.0], 22),
            system("octas")]
    s = W.merge(reps)
    errs, ref, _ = compare_forces(dem, s, precision, decomp=DECOMPS[decomp])
    assert_parity(errs, precision, f"batched/{decomp}")


@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
def test_nlist_growth(dem, precision):
    """A neighbour list far too small must grow transparently."""
    s = system("cubes")
    errs, _, _ = compare_forces(dem, s, precision, nlist_cap=2)
    assert_parity(errs, precision, "nlist_cap=2")


def test_no_contacts_exact_zero(dem):
    """Particles farther apart than the interaction range get exactly zero."""
    sh = W.cube(1.0, 0.15)
    pos = W.sc_sites([4, 4, 4], [2.2] * 3)
    n = len(pos)
    s = W.System(3, [sh], np.zeros(n, np.int32), pos, W.random_quaternions(np.random.default_rng(0), n),
                 np.zeros((n, 3)), np.zeros((n, 3)), np.full((1, 3), 8.8), np.array([n], np.int32),
                 1.0, 0.3)
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        f, t = d.forces()
        U, _, _ = d.energy()
    assert np.all(f == 0.0) and np.all(t == 0.0) and U[0] == 0.0


@pytest.mark.parametrize("decomp", list(DECOMPS))
def test_deterministic(dem, decomp):
    s = system("mixed3d")
    outs = []
    for _ in range(2):
        with dem.DEM(s, dem.DEM_FP32_COMP, decomp=DECOMPS[decomp]) as d:
            outs.append(d.forces())
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_compensated_not_worse(dem):
    """Two-sum accumulation is at least as close to the oracle as plain FP32."""
    s = system("cubes")
    e1, _, _ = compare_forces(dem, s, 1)
    e2, _, _ = compare_forces(dem, s, 2)
    assert e2["normF"] <= e1["normF"] * 1.05 + 1e-12


def test_device_pointer_state(dem):
    """State passed as CUDA torch tensors on torch's stream (device_ptrs=1)."""
    import torch
    s = system("cubes")
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        f_host, _ = d.forces()
        stream = torch.cuda.current_stream()
        dem.dem_set_stream(d.ctx, stream.cuda_stream)
        dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
        dem.dem_set_state(d.ctx, dev(s.shape_id, torch.int32), dev(s.pos), dev(s.orient), dev(s.vel),
                          dev(s.angmom), device_ptrs=1)
        f_dev = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
        t_dev = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
        dem.dem_get_forces(d.ctx, f_dev, t_dev, device_ptrs=1)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(f_dev.cpu().numpy(), f_host)


def test_state_roundtrip(dem):
    s = system("prisms")
    with dem.DEM(s, dem.DEM_FP64) as d:
        st = d.state()
    np.testing.assert_allclose(st["pos"], np.mod(s.pos, s.box[0]), atol=1e-12)
    np.testing.assert_allclose(st["vel"], s.vel, atol=0)
    qn = s.orient / np.linalg.norm(s.orient, axis=1, keepdims=True)
    np.testing.assert_allclose(st["orient"], qn, atol=1e-15)
    np.testing.assert_allclose(st["angmom"], s.angmom, atol=1e-13)


def _ctx_errors(d, system):
    """Errors of a live context's current outputs against the oracle."""
    import oracle
    f, t = d.forces()
    U, _, _ = d.energy()
    out = dict(force=f, torque=t, U=U, W=d.virial(), energy=d.particle_energy(), counts=None)
    return force_errors(system, oracle.forces(system), out)


@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
def test_set_state_keeps_valid_list(dem, precision):
    """A state upload with the same shapes keeps the neighbour list while
    every particle is within skin/2 of its position at the build, and
    rebuilds it otherwise; new shape ids rebuild everything.  Forces match
    the oracle in every case."""
    s = system("cubes")
    rng = np.random.default_rng(41)
    with dem.DEM(s, precision) as d:
        skin = d.get_param("skin")
        rb = lambda: int(d.counters()[13])
        r0 = rb()
        # small moves: the list stays
        small = s.pos + rng.uniform(-1, 1, s.pos.shape) * 0.2 * skin / np.sqrt(3)
        t = W.System(s.dim, s.shapes, s.shape_id, np.mod(small, s.box[0]), s.orient, s.vel,
                     s.angmom, s.box, s.replica_sizes, s.epsilon, s.sigma)
        dem.dem_set_state(d.ctx, t.shape_id, t.pos, t.orient, t.vel, t.angmom)
        assert rb() == r0, "a valid list must be kept"
        assert_parity(_ctx_errors(d, t), precision, "set_state small move")
        # one particle beyond skin/2: rebuilt
        big = small.copy()
        big[7] += 0.8 * skin
        t.pos = np.mod(big, s.box[0])
        dem.dem_set_state(d.ctx, t.shape_id, t.pos, t.orient, t.vel, t.angmom)
        assert rb() == r0 + 1, "the list must be rebuilt"
        assert_parity(_ctx_errors(d, t), precision, "set_state large move")
    # new shape ids: full setup (a cube becomes a smaller cube)
    s2 = system("dented")
    with dem.DEM(s2, precision) as d:
        ids = s2.shape_id.copy()
        ids[ids == 0] = 1            # dented cubes become cubes
        t = W.System(s2.dim, s2.shapes, ids, s2.pos, s2.orient, s2.vel, s2.angmom, s2.box,
                     s2.replica_sizes, s2.epsilon, s2.sigma)
        dem.dem_set_state(d.ctx, t.shape_id, t.pos, t.orient, t.vel, t.angmom)
        # the spheres nested in the dents now lie inside plain cubes: an
        # overlapping state, compared on the term scales only
        assert_parity(_ctx_errors(d, t), precision, "set_state new shapes", rel=False)


@pytest.mark.parametrize("group", [4, 8, 16, 32])
@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "fp32c"])
@pytest.mark.parametrize("name", ["mixed3d", "polys2d", "dented"])
def test_split_group_sizes(dem, name, precision, group):
    """SPLIT with each number of particles per warp: parity with the oracle
    and the same work as the THREAD decomposition."""
    s = system(name)
    errs, ref, out = compare_forces(dem, s, precision, decomp=4, split_group=group)
    assert_parity(errs, precision, f"{name}/split group {group}")
    with dem.DEM(s, dem.DEM_FP64, decomp=4, split_group=group) as d:
        assert d.get_param("split_group") == group
        c_split = d.counters()
        for bad in (1, 2, 12, 64, 8.5, -4):
            with pytest.raises(dem.DemError):
                d.set_param("split_group", bad)
    with dem.DEM(s, dem.DEM_FP64, decomp=1) as d:
        c_thread = d.counters()
    keep = [k for k in range(18) if k not in (3, 13, 14)]
    np.testing.assert_array_equal(c_split[keep], c_thread[keep])


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp32", "fp32c"])
@pytest.mark.parametrize("name", ["mixed3d", "polys2d"])
def test_split_slices(dem, name, precision):
    """SPLIT run slice after slice (parameter split_slice): parity with the
    oracle, and the same forces as one pass (each particle's terms keep their
    order: the kind order within a warp's pool does not depend on the other
    particles of the pool while a pool fits one chunk)."""
    s = system(name)
    errs, ref, out = compare_forces(dem, s, precision, decomp=4, split_slice=64)
    assert_parity(errs, precision, f"{name}/split slices")
    res = []
    for sl in (0, 64, 96):
        with dem.DEM(s, precision, decomp=4, split_slice=sl, persistent=0) as d:
            res.append(d.forces())
            d.step(10, 1e-3, dem.DEM_NVE)   # the step path (graph) with slices
            assert np.isfinite(d.energy()[2]).all()
    for f, t in res[1:]:
        np.testing.assert_array_equal(f, res[0][0])
        np.testing.assert_array_equal(t, res[0][1])
