"""GPU dynamics against the FP64 oracle's integrator (velocity Verlet, body-
axis free-rotor splitting, Nose-Hoover Trotter split), through the C ABI.

* FP64 mode: trajectories (positions, velocities, orientations, angular
  momenta, thermostat variables) match the oracle after 100 steps to 1e-9
  (absolute, lengths in edge units) in 3D and 2D, NVE and NVT, one or several
  replicas.  Over 100 steps of a dense cluster, chaotic growth amplifies
  rounding differences of order 1e-16 by far less than 1e7.
* FP32 modes: the same within 1e-4 after 100 steps.
* Energy: the NVE energy error scales as dt^2 (Section "Energy
  Conservation"); the NVT extended energy is conserved.
* The captured-graph path equals the launch-by-launch path bit for bit, and
  a neighbour-list overflow retried from the start of the call gives the
  same trajectory bit for bit (here through the cooperative multi-step
  kernel, the default for systems this small).
* Every trajectory case runs the step kernels with three decompositions and
  the cooperative multi-step kernel.
"""
import numpy as np
import pytest

import oracle
from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import load_dem
from tests.helpers import dent_points, nest_guests, notch_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _cluster(shapes, n, box, seed, **kw):
    rng = np.random.default_rng(seed)
    return W.contact_cluster(shapes, np.zeros(n, np.int32) if len(shapes) == 1
                             else np.arange(n) % len(shapes), box, rng, **kw)


def _min_image(d, box):
    return d - box * np.round(d / box)


def _compare_states(s, st, ref, tol_x, tol_v):
    for r, sl in enumerate(s.replica_slices()):
        dx = _min_image(st["pos"][sl] - ref["pos"][sl], s.box[r])
        assert np.abs(dx).max() < tol_x, f"positions differ by {np.abs(dx).max():.3e}"
    assert np.abs(st["vel"] - ref["vel"]).max() < tol_v
    assert np.abs(st["angmom"] - ref["angmom"]).max() < tol_v
    if s.dim == 3:
        q1, q2 = st["orient"], ref["orient"]
        dq = np.minimum(np.abs(q1 - q2).max(1), np.abs(q1 + q2).max(1))
        assert dq.max() < tol_x, f"orientations differ by {dq.max():.3e}"
    else:
        dth = np.angle(np.exp(1j * (st["orient"][:, 0] - ref["orient"][:, 0])))
        assert np.abs(dth).max() < tol_x


CASES = {
    "cubes_nve": (lambda: _cluster([W.cube(1.0, 0.15)], 64, [9.0] * 3, 31, sigma=0.3), "nve"),
    "cubes_nvt": (lambda: _cluster([W.cube(1.0, 0.15)], 64, [9.0] * 3, 32, sigma=0.3), "nvt"),
    "mixed_nvt": (lambda: _cluster([W.tetrahedron(1.0, 0.15), W.triangular_prism(1.0, 1.0, 0.1),
                                    W.octahedron(0.8, 0.12)], 60, [9.0] * 3, 33), "nvt"),
    "squares_nve": (lambda: _cluster([W.square(1.0, 0.15)], 80, [16.0, 16.0], 34, sigma=0.3), "nve"),
    "polys_nvt": (lambda: _cluster([W.polygon(6, 0.6, 0.12), W.square(0.9, 0.1)], 80,
                                   [16.0, 16.0], 35), "nvt"),
    # concave inner shapes (Section "Model")
    "dented_nvt": (lambda: nest_guests(_cluster([W.dented_cube(1.0, 0.6, 0.12)], 50, [9.0] * 3, 36),
                                       range(0, 50, 2), W.sphere(0.15, 0.009),
                                       dent_points(W.dented_cube(1.0, 0.6, 0.12), 0.27), 36), "nvt"),
    "lshapes_nve": (lambda: nest_guests(_cluster([W.l_shape2d(0.6, 0.12)], 70, [16.0, 16.0], 37),
                                        range(0, 70, 2), W.disk(0.15, 0.01),
                                        notch_points(W.l_shape2d(0.6, 0.12), 0.27), 37), "nve"),
}


# the step kernels with three pair-kernel decompositions, and the cooperative
# multi-step kernel
MODES = {"thread": {"decomp": 1, "persistent": 0}, "staged": {"decomp": 3, "persistent": 0},
         "split": {"decomp": 4, "persistent": 0}, "persistent": {"persistent": 1}}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (2, 1e-4), (1, 1e-4)],
                         ids=["fp64", "fp32c", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_trajectory_matches_oracle(dem, name, precision, tol, mode):
    mk, ens = CASES[name]
    s = mk()
    n, dt = 100, 1e-3
    ref, tr = oracle.run(s, n, dt, ensemble=ens, kT=1.0, tau=0.5)
    assert tr[0, :, 2].max() > 0.1, "the run must have interactions"
    with dem.DEM(s, precision, **MODES[mode]) as d:
        d.step(n, dt, dem.DEM_NVT if ens == "nvt" else dem.DEM_NVE, kT=1.0, tau_T=0.5)
        assert d.get_param("persistent_used") == (mode == "persistent")
        st = d.state()
        U, K, H = d.energy()
    _compare_states(s, st, ref, tol, 10 * tol)
    if ens == "nvt":
        assert np.abs(st["thermo"] - ref["thermo"]).max() < 10 * tol
    assert H[0] == pytest.approx(tr[0, -1, 3], rel=1e-9 if precision == 0 else 1e-4)


def test_multi_replica_nvt_fp64(dem):
    reps = [_cluster([W.cube(1.0, 0.15)], 40, [8.0] * 3, 41),
            _cluster([W.tetrahedron(1.0, 0.2)], 70, [8.0] * 3, 42),
            _cluster([W.triangular_prism(1.0, 1.0, 0.15)], 25, [6.0] * 3, 43)]
    s = W.merge(reps)
    ref, tr = oracle.run(s, 100, 1e-3, ensemble="nvt", kT=1.5, tau=0.3)
    with dem.DEM(s, dem.DEM_FP64) as d:
        d.step(60, 1e-3, dem.DEM_NVT, kT=1.5, tau_T=0.3)
        d.step(40, 1e-3, dem.DEM_NVT, kT=1.5, tau_T=0.3)   # two calls = one run
        st = d.state()
    _compare_states(s, st, ref, 1e-9, 1e-8)
    assert np.abs(st["thermo"] - ref["thermo"]).max() < 1e-8


def test_energy_error_scales_dt2(dem):
    s = _cluster([W.cube(1.0, 0.15)], 60, [12.0] * 3, 51, sigma=0.3, gap=(0.95, 1.1), gap_min=0.9)
    errs = []
    for dt in (2e-3, 1e-3):
        with dem.DEM(s, dem.DEM_FP64) as d:
            _, _, H0 = d.energy()
            dev = 0.0
            for _ in range(int(round(0.2 / dt / 10))):
                d.step(10, dt, dem.DEM_NVE)
                dev = max(dev, abs(d.energy()[2][0] - H0[0]))
        errs.append(dev)
    assert 2.5 < errs[0] / errs[1] < 6.0, errs


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "fp32c"])
def test_nvt_conserved_quantity(dem, precision):
    # the oracle's own run of this input drifts by 4.5e-4 K over the same steps
    s = _cluster([W.cube(1.0, 0.15)], 80, [12.0] * 3, 52, sigma=0.3, gap=(1.0, 1.12), gap_min=0.98)
    with dem.DEM(s, precision) as d:
        d.step(1, 1e-3, dem.DEM_NVT, kT=1.0, tau_T=0.5)
        H = []
        for _ in range(40):
            d.step(25, 1e-3, dem.DEM_NVT, kT=1.0, tau_T=0.5)
            H.append(d.energy()[2][0])
        K = d.energy()[1][0]
    assert np.ptp(H) < 2e-3 * K


def test_graph_equals_eager(dem):
    s = _cluster([W.cube(1.0, 0.15)], 150, [14.0] * 3, 53, sigma=0.3, gap=(0.95, 1.1), gap_min=0.9)
    out = []
    for graph in (1, 0):
        with dem.DEM(s, dem.DEM_FP32_COMP, graph=graph, persistent=0) as d:
            d.step(50, 1e-3, dem.DEM_NVT, kT=1.0, tau_T=0.5)
            out.append(d.state())
    for k in ("pos", "vel", "orient", "angmom", "thermo"):
        np.testing.assert_array_equal(out[0][k], out[1][k])


@pytest.mark.parametrize("ens", ["nve", "nvt"])
def test_graph_eager_profiling(dem, ens):
    """Steps replayed from the captured graph and launched directly, with
    the pair-kernel profiling (CUDA events around the pair kernels: graph
    event nodes, or plain records) on and off, in calls of several lengths,
    give identical trajectories, and the profiled totals cover every step."""
    small = _cluster([W.cube(1.0, 0.15)], 150, [14.0] * 3, 55, sigma=0.3, gap=(0.95, 1.1),
                     gap_min=0.9)
    e = dem.DEM_NVE if ens == "nve" else dem.DEM_NVT
    out = []
    for graph, prof in ((1, 0), (1, 1), (0, 1), (0, 0)):
        with dem.DEM(small, dem.DEM_FP32_COMP, graph=graph, persistent=0) as d:
            d.set_param("profile", prof)
            for n in (7, 1, 12):
                d.step(n, 1e-3, e, kT=1.0, tau_T=0.5)
            if prof:
                assert d.get_param("pair_launches") == 20
                assert d.get_param("pair_ms_total") > 0
            out.append(d.state())
    for o in out[1:]:
        for k in ("pos", "vel", "orient", "angmom", "thermo"):
            np.testing.assert_array_equal(o[k], out[0][k])


def test_overflow_retry_same_trajectory(dem):
    s = _cluster([W.cube(1.0, 0.15)], 150, [14.0] * 3, 54, sigma=0.3, gap=(0.95, 1.1), gap_min=0.9)
    out = []
    for cap in (None, 3):
        params = {} if cap is None else {"nlist_cap": cap}
        with dem.DEM(s, dem.DEM_FP32_COMP, **params) as d:
            d.step(80, 1e-3, dem.DEM_NVE)
            out.append(d.state())
            if cap:
                assert d.get_param("nlist_cap") > cap
    for k in ("pos", "vel", "orient", "angmom"):
        np.testing.assert_array_equal(out[0][k], out[1][k])


def test_set_box_compresses(dem):
    s = W.config_cubes_4096(n_side=6)
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        st0 = d.state()
        new = s.box * 0.97
        d.set_box(new)
        st1 = d.state()
        np.testing.assert_allclose(st1["pos"], st0["pos"] * 0.97, rtol=1e-14, atol=1e-13)
        d.step(20, 1e-3, dem.DEM_NVT, kT=1.0, tau_T=0.5)
        assert np.isfinite(d.energy()[2]).all()
