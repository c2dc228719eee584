"""The cooperative multi-step kernel of dem_step (parameter "persistent"),
through the C ABI.

* It runs the per-step phases of the step kernels (first half step, pair
  terms of Eq. DEM / Eq. DEM_2D per list entry, per-particle sums in list
  order, second half step, Nose-Hoover thermostat) in one launch with
  grid-wide barriers: the trajectory equals the step kernels' with the WARP
  decomposition bit for bit in the FP32 modes, and to 1e-11 in FP64 (the
  compiler fuses some multiply-adds of the FP64 free rotor differently in
  the two kernels), in 2D and 3D, NVE and NVT, with list rebuilds inside the
  call, replicas summed directly and by chunks, and calls of several
  lengths.
* Against the FP64 oracle's integrator it meets the trajectory bars of the
  step kernels.
* Its barrier waits are bounded: a launch in which one block never arrives
  returns DEM_ERR_TIMEOUT after the limit, the state is that of the start of
  the call, and the context steps on as before.
* A long call launches far fewer kernels than it runs steps.
"""
import numpy as np
import pytest

import oracle
from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import load_dem

pytestmark = pytest.mark.gpu

KEYS = ("pos", "vel", "orient", "angmom", "thermo")


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _cluster(shapes, n, box, seed, **kw):
    rng = np.random.default_rng(seed)
    return W.contact_cluster(shapes, np.zeros(n, np.int32) if len(shapes) == 1
                             else np.arange(n) % len(shapes), box, rng, **kw)


SYSTEMS = {
    "cubes": lambda: _cluster([W.cube(1.0, 0.15)], 150, [14.0] * 3, 61, sigma=0.3,
                              gap=(0.95, 1.1), gap_min=0.9),
    "mixed": lambda: _cluster([W.tetrahedron(1.0, 0.15), W.triangular_prism(1.0, 1.0, 0.1),
                               W.octahedron(0.8, 0.12)], 120, [11.0] * 3, 62),
    "squares": lambda: _cluster([W.square(1.0, 0.15)], 200, [26.0, 26.0], 63, sigma=0.3),
    "replicas": lambda: W.merge([_cluster([W.cube(1.0, 0.15)], 60, [9.0] * 3, 64, sigma=0.3),
                                 _cluster([W.tetrahedron(1.0, 0.2)], 90, [9.0] * 3, 65)]),
}


def _run(dem, s, precision, ens, persistent, calls=(23, 1, 76), dt=2e-3):
    e = dem.DEM_NVT if ens == "nvt" else dem.DEM_NVE
    with dem.DEM(s, precision, decomp=dem.DEM_DECOMP_WARP, persistent=persistent) as d:
        r0 = int(d.counters()[13])
        for n in calls:
            d.step(n, dt, e, kT=1.0, tau_T=0.5)
        used = d.get_param("persistent_used")
        st = d.state()
        U, K, H = d.energy()
        st["U"], st["H"] = U, H
        st["rebuilds"] = int(d.counters()[13]) - r0
    return st, used


@pytest.mark.parametrize("ens", ["nve", "nvt"])
@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp32", "fp32c"])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_persistent_equals_warp_steps(dem, name, precision, ens):
    s = SYSTEMS[name]()
    ref, used0 = _run(dem, s, precision, ens, 0)
    got, used1 = _run(dem, s, precision, ens, 1)
    assert used0 == 0 and used1 == 1
    assert ref["rebuilds"] > 0, "the run must rebuild its list inside the calls"
    assert got["rebuilds"] == ref["rebuilds"]
    for k in KEYS + ("U", "H"):
        if precision == 0:
            np.testing.assert_allclose(got[k], ref[k], rtol=0, atol=1e-11 * (1 + np.abs(ref[k]).max()),
                                       err_msg=k)
        else:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_persistent_chunked_replica_nvt(dem):
    """A replica of more than 2048 particles: the thermostat sums by chunks
    and the second scaling is a separate per-particle phase."""
    s = W.config_cubes_4096(n_side=14)
    assert s.n > 2048
    ref, _ = _run(dem, s, dem.DEM_FP32_COMP, "nvt", 0, calls=(15, 10), dt=1e-3)
    got, used = _run(dem, s, dem.DEM_FP32_COMP, "nvt", 1, calls=(15, 10), dt=1e-3)
    assert used == 1
    for k in KEYS + ("U", "H"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (2, 1e-4)], ids=["fp64", "fp32c"])
@pytest.mark.parametrize("ens", ["nve", "nvt"])
def test_persistent_matches_oracle(dem, ens, precision, tol):
    s = _cluster([W.cube(1.0, 0.15)], 64, [9.0] * 3, 66, sigma=0.3)
    n, dt = 100, 1e-3
    ref, tr = oracle.run(s, n, dt, ensemble=ens, kT=1.0, tau=0.5)
    assert tr[0, :, 2].max() > 0.1
    with dem.DEM(s, precision, persistent=1) as d:
        d.step(n, dt, dem.DEM_NVT if ens == "nvt" else dem.DEM_NVE, kT=1.0, tau_T=0.5)
        assert d.get_param("persistent_used") == 1
        st = d.state()
    dx = st["pos"] - ref["pos"]
    dx -= s.box[0] * np.round(dx / s.box[0])
    assert np.abs(dx).max() < tol
    assert np.abs(st["vel"] - ref["vel"]).max() < 10 * tol
    assert np.abs(st["angmom"] - ref["angmom"]).max() < 10 * tol
    if ens == "nvt":
        assert np.abs(st["thermo"] - ref["thermo"]).max() < 10 * tol


@pytest.mark.parametrize("ens", ["nve", "nvt"])
def test_persistent_timeout_restores_state(dem, ens):
    # FP64: the restored state's forces, taken on a freshly built list, equal
    # the ones taken on the list of the interrupted run (in the FP32 modes the
    # list's stored separations round differently)
    s = SYSTEMS["cubes"]()
    e = dem.DEM_NVT if ens == "nvt" else dem.DEM_NVE
    with dem.DEM(s, dem.DEM_FP64, decomp=dem.DEM_DECOMP_WARP, persistent=1) as d:
        d.step(10, 1e-3, e, kT=1.0, tau_T=0.5)
        before = d.state()
        f0, t0 = d.forces()
        d.set_param("persistent_wait_ms", 20)
        d.set_param("persistent_test_stall", 1)
        with pytest.raises(dem.DemError) as ei:
            d.step(10, 1e-3, e, kT=1.0, tau_T=0.5)
        assert ei.value.code == dem.DEM_ERR_TIMEOUT
        after = d.state()
        for k in KEYS:
            np.testing.assert_array_equal(after[k], before[k], err_msg=k)
        f1, t1 = d.forces()
        np.testing.assert_array_equal(f1, f0)
        # the context steps on: the same 20 steps as an undisturbed run
        d.set_param("persistent_wait_ms", 1000)
        d.step(20, 1e-3, e, kT=1.0, tau_T=0.5)
        got = d.state()
    with dem.DEM(s, dem.DEM_FP64, decomp=dem.DEM_DECOMP_WARP, persistent=1) as d:
        d.step(10, 1e-3, e, kT=1.0, tau_T=0.5)
        d.step(20, 1e-3, e, kT=1.0, tau_T=0.5)
        ref = d.state()
    for k in KEYS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_persistent_launches(dem):
    s = SYSTEMS["squares"]()
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:       # the default: on for small systems
        l0 = d.get_param("launches")
        d.step(400, 1e-3, dem.DEM_NVT, kT=1.0, tau_T=0.5)
        assert d.get_param("persistent_used") == 1
        per_step = (d.get_param("launches") - l0) / 400
    assert per_step < 1.0, per_step


def test_persistent_param_checks(dem):
    s = SYSTEMS["cubes"]()
    with dem.DEM(s, dem.DEM_FP32) as d:
        for bad in (-2, 2):
            with pytest.raises(dem.DemError):
                d.set_param("persistent", bad)
        with pytest.raises(dem.DemError):
            d.set_param("persistent_wait_ms", 0.5)
        # profiling times the pair kernels of the step kernels: no cooperative launch
        d.set_param("persistent", 1)
        d.set_param("profile", 1)
        d.step(3, 1e-3, dem.DEM_NVE)
        assert d.get_param("persistent_used") == 0
        d.set_param("profile", 0)
        d.step(3, 1e-3, dem.DEM_NVE)
        assert d.get_param("persistent_used") == 1


@pytest.mark.parametrize("name", ["squares", "cubes"])
def test_autotune_times_both_paths(dem, name):
    """dem_autotune times a few steps with the per-step kernels and with the
    cooperative kernel, keeps the faster for dem_step and leaves the state as
    it found it."""
    s = SYSTEMS[name]()
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        d.step(5, 1e-3, dem.DEM_NVT, kT=1.0, tau_T=0.5)
        before = d.state()
        dem.dem_autotune(d.ctx)
        after = d.state()
        for k in KEYS:
            np.testing.assert_array_equal(after[k], before[k], err_msg=k)
        tg, tp = d.get_param("autotune_step_ms_graph"), d.get_param("autotune_step_ms_persistent")
        assert tg > 0 and tp > 0
        choice = d.get_param("persistent_auto")
        assert choice == (1 if tp < tg else 0)
        d.step(5, 1e-3, dem.DEM_NVT, kT=1.0, tau_T=0.5)
        assert d.get_param("persistent_used") == choice
