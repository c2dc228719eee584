"""GPU parity of the isotropic barostat (DEM_NPT) against the FP64 oracle,
through the C ABI.

Inputs: seeded contact-rich periodic clusters of cubes and of mixed shapes
whose boxes move by several percent over the run.  Checks: trajectories,
thermostat / barostat variables and boxes against oracle.run(ensemble="npt")
(FP64 to 1e-9, FP32 modes to 1e-4); FP64 runs identical for any chunking
of the call (the cell grids and the list follow the box between chunks);
forces after a strong compression equal to the oracle's at that state (the
scaled list separations and the rebuild pad miss no pair); the conserved
quantity; argument errors.
"""
import numpy as np
import pytest

import oracle
from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import TOL, load_dem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _cluster(shapes, n, box, seed, **kw):
    rng = np.random.default_rng(seed)
    ids = np.arange(n) % len(shapes)
    return W.contact_cluster(shapes, ids.astype(np.int32), box, rng, gap=(0.95, 1.12),
                             gap_min=0.92, free=0.0, **kw)


CASES = {
    "cubes": lambda: _cluster([W.cube(1.0, 0.15)], 90, [9.0] * 3, 61, sigma=0.3),
    "mixed": lambda: _cluster([W.cube(1.0, 0.15), W.tetrahedron(1.0, 0.15),
                               W.octahedron(0.8, 0.12)], 80, [9.0] * 3, 62),
}
PRESSURE = {"cubes": 1.0, "mixed": 0.4}     # boxes move by 1-12% in volume in 100 steps


def _run(dem, s, precision, n, dt, P, tau_P, **params):
    with dem.DEM(s, precision, **params) as d:
        d.set_barostat(P, tau_P)
        d.step(n, dt, dem.DEM_NPT, kT=1.0, tau_T=0.5)
        st = d.state()
        U, K, H = d.energy()
    return st, U, K, H


def _compare(s, st, ref, tol):
    L = ref["box"]
    np.testing.assert_allclose(st["box"], L, rtol=tol, atol=0)
    for r, sl in enumerate(s.replica_slices()):
        d = st["pos"][sl] - ref["pos"][sl]
        d -= L[r] * np.round(d / L[r])
        assert np.abs(d).max() < tol * 10, ("pos", np.abs(d).max())
    np.testing.assert_allclose(st["vel"], ref["vel"], atol=10 * tol)
    qd = np.minimum(np.abs(st["orient"] - ref["orient"]).max(1),
                    np.abs(st["orient"] + ref["orient"]).max(1))
    assert qd.max() < 10 * tol
    np.testing.assert_allclose(st["angmom"], ref["angmom"], atol=10 * tol * max(1.0, np.abs(ref["angmom"]).max()))
    np.testing.assert_allclose(st["thermo"], ref["thermo"], atol=10 * tol * max(1.0, np.abs(ref["thermo"]).max()))


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (2, 1e-4)], ids=["fp64", "fp32c"])
@pytest.mark.parametrize("name", list(CASES))
def test_npt_trajectory_matches_oracle(dem, name, precision, tol):
    s = CASES[name]()
    n, dt, P, tau_P = 100, 1e-3, PRESSURE[name], 0.5
    ref, tr = oracle.run(s, n, dt, ensemble="npt", kT=1.0, tau=0.5, P=P, tau_P=tau_P)
    assert tr[0, :, 2].max() > 0.1, "the run must have interactions"
    assert abs(tr[0, -1, 4] / np.prod(s.box[0]) - 1.0) > 0.01, "the box must move"
    st, U, K, H = _run(dem, s, precision, n, dt, P, tau_P, npt_chunk=30)
    _compare(s, st, ref, tol)
    assert H[0] == pytest.approx(tr[0, -1, 3], rel=1e-9 if precision == 0 else 1e-4)


def test_npt_chunking_does_not_change_fp64(dem):
    s = CASES["cubes"]()
    a = _run(dem, s, dem.DEM_FP64, 60, 1e-3, 1.0, 0.5, npt_chunk=60)[0]
    b = _run(dem, s, dem.DEM_FP64, 60, 1e-3, 1.0, 0.5, npt_chunk=7)[0]
    for k in ("pos", "vel", "orient", "angmom", "thermo", "box"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "fp32c"])
def test_forces_after_compression(dem, precision):
    """A strong compression (volume down by ~20%) inside one call chunk, so
    that the last forces come from a list built in a larger box: they equal
    the oracle's at the final state (no pair missed, separations scaled
    right)."""
    s = CASES["mixed"]()
    with dem.DEM(s, precision, npt_chunk=400) as d:
        d.set_barostat(0.75, 0.5)
        d.step(300, 1e-3, dem.DEM_NPT, kT=1.0, tau_T=0.5)
        st = d.state()
        f, tq = d.forces()
    assert np.prod(st["box"][0]) < 0.9 * np.prod(s.box[0])
    t = W.System(s.dim, s.shapes, s.shape_id, st["pos"], st["orient"], st["vel"], st["angmom"],
                 st["box"], s.replica_sizes, s.epsilon, s.sigma)
    ref = oracle.forces(t)
    live = (ref["flags"] == 0) & (ref["fscale"] > 0)
    assert live.sum() >= 8, "the final state must have contacts"
    errF = np.linalg.norm(f - ref["force"], axis=1)[live] / ref["fscale"][live]
    assert errF.max() < TOL[precision], errF.max()
    assert np.all(f[ref["fscale"] == 0] == 0.0)


def test_npt_conserved_quantity(dem):
    s = CASES["cubes"]()
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        d.set_barostat(1.0, 0.5)
        H = []
        for _ in range(10):
            d.step(50, 1e-3, dem.DEM_NPT, kT=1.0, tau_T=0.5)
            H.append(d.energy()[2][0])
        K = d.energy()[1][0]
    assert np.ptp(H) < 5e-3 * K, (np.ptp(H), K)


def test_npt_arguments(dem):
    s = CASES["cubes"]()
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        with pytest.raises(dem.DemError):
            d.step(1, 1e-3, dem.DEM_NPT, kT=1.0, tau_T=0.5)      # no barostat set
        with pytest.raises(dem.DemError):
            d.set_barostat(-1.0, 0.5)
        with pytest.raises(dem.DemError):
            d.set_barostat(1.0, 0.0)
