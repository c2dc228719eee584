"""Failure detection injected on the host (no GPU fault, no device-side
injector): invalid states handed to dem_set_state, from host and device
arrays, and a state whose forces are not finite.

* a non-finite position, velocity, angular momentum or orientation, or a
  quaternion of zero norm, is found on the device as the arrays are
  imported and returns DEM_ERR_ARG; the kernels that follow in the same
  call run on a harmless substitute state;
* two coincident particles give non-finite forces: DEM_ERR_NONFINITE;
* after either error the context has no state (dem_step returns
  DEM_ERR_STATE), and a valid dem_set_state makes it usable again, with
  forces matching the oracle;
* a term buffer too small for the FP32 + two-sum SPLIT evaluation (one
  record per warp) overflows: the evaluation is redone with a larger
  buffer and gives the same forces and trajectory as one that never
  overflowed.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import TOL, assert_parity, force_errors, load_dem
from tests.helpers import copy_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _system(dim):
    rng = np.random.default_rng(5 + dim)
    if dim == 3:
        return W.contact_cluster([W.cube(1.0, 0.15)], np.zeros(120, np.int32), [12.0] * 3, rng,
                                 sigma=0.3)
    return W.contact_cluster([W.square(1.0, 0.15)], np.zeros(120, np.int32), [25.0] * 2, rng,
                             sigma=0.3)


def _set(dem, d, s, device):
    arrs = [s.shape_id, s.pos, s.orient, s.vel, s.angmom]
    if device:
        import torch
        arrs = [torch.as_tensor(np.ascontiguousarray(a), device="cuda",
                                dtype=torch.int32 if k == 0 else torch.float64)
                for k, a in enumerate(arrs)]
    dem.dem_set_state(d.ctx, *arrs, device_ptrs=1 if device else 0)


def _check_recovers(dem, d, s, precision):
    import oracle
    _set(dem, d, s, False)
    f, t = d.forces()
    U, K, H = d.energy()
    ref = oracle.forces(s)
    out = dict(force=f, torque=t, U=U, W=d.virial(), energy=d.particle_energy(), counts=None)
    assert_parity(force_errors(s, ref, out), precision, "recovered")
    d.step(5, 1e-3, dem.DEM_NVE)


BAD = {
    "pos_nan": ("pos", 7, 0, np.nan),
    "pos_inf": ("pos", 0, 1, np.inf),
    "vel_inf": ("vel", 33, 0, -np.inf),
    "angmom_nan": ("angmom", 119, 0, np.nan),
    "orient_nan": ("orient", 50, 0, np.nan),
    "orient_zero": ("orient", 61, None, 0.0),
}


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("case", list(BAD))
def test_bad_input_rejected(dem, case, dim, device):
    s = _system(dim)
    field, i, comp, val = BAD[case]
    if case == "orient_zero" and dim == 2:
        pytest.skip("2D orientations are angles: every finite angle is valid")
    bad = copy_system(s)
    arr = getattr(bad, field)
    if comp is None:
        arr[i, :] = val
    else:
        arr[i, comp % arr.shape[1]] = val
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        with pytest.raises(dem.DemError) as ei:
            _set(dem, d, bad, device)
        assert ei.value.code == dem.DEM_ERR_ARG
        assert f"particle {i}" in str(ei.value)
        with pytest.raises(dem.DemError) as ei:
            d.step(1, 1e-3, dem.DEM_NVE)
        assert ei.value.code == dem.DEM_ERR_STATE
        _check_recovers(dem, d, s, dem.DEM_FP32_COMP)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_coincident_particles_nonfinite(dem, precision):
    """Two particles with the same centre and orientation: nearest-point
    distances of zero, non-finite WCA terms, DEM_ERR_NONFINITE."""
    s = _system(3)
    bad = copy_system(s)
    bad.pos[1] = bad.pos[0]
    bad.orient[1] = bad.orient[0]
    with dem.DEM(s, precision) as d:
        with pytest.raises(dem.DemError) as ei:
            _set(dem, d, bad, False)
        assert ei.value.code == dem.DEM_ERR_NONFINITE
        with pytest.raises(dem.DemError) as ei:
            d.step(1, 1e-3, dem.DEM_NVE)
        assert ei.value.code == dem.DEM_ERR_STATE
        _check_recovers(dem, d, s, precision)


def test_noalloc_rejects_nonfinite(dem):
    import torch
    s = _system(3)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    pos = s.pos.copy()
    pos[3, 2] = np.nan
    f = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dem.DemError) as ei:
        dem.dem_forces_noalloc(s.shapes, s.epsilon, s.sigma, s.box[0],
                               dev(s.shape_id, torch.int32), dev(pos, torch.float64),
                               dev(s.orient, torch.float64), 2, f, t)
    assert ei.value.code == dem.DEM_ERR_ARG and "particle 3" in str(ei.value)


@pytest.mark.parametrize("dim", [3, 2])
def test_term_buffer_overflow_retry(dem, dim):
    import oracle
    s = _system(dim)
    out = []
    for cap in (None, 1):
        params = {"decomp": dem.DEM_DECOMP_SPLIT, "persistent": 0}
        if cap:
            params["term_cap"] = cap
        with dem.DEM(s, dem.DEM_FP32_COMP, **params) as d:
            f, t = d.forces()
            e = d.particle_energy()
            if cap:
                assert d.get_param("term_cap") > cap
                out_o = dict(force=f, torque=t, U=d.energy()[0], W=d.virial(), energy=e,
                             counts=None)
                assert_parity(force_errors(s, oracle.forces(s), out_o), dem.DEM_FP32_COMP,
                              f"term overflow {dim}d")
                d.set_param("term_cap", 1)          # overflow again inside a step call
            d.step(30, 1e-3, dem.DEM_NVE)
            out.append((f, t, e, d.state()))
    for k in range(3):
        np.testing.assert_array_equal(out[1][k], out[0][k])
    for k in ("pos", "vel", "orient", "angmom"):
        np.testing.assert_array_equal(out[1][3][k], out[0][3][k])
