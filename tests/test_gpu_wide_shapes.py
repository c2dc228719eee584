"""Shapes with more than 32 vertices, edges or faces (up to 128 of each):
the 80-face icosphere (42 V / 120 E / 80 F) and a 100-gon, whose feature
masks take the two-level form (four 32-bit words, empty words skipped).
Contexts holding such a shape run the THREAD decomposition; the tests check
parity with the FP64 oracle in every precision, alone and mixed with
one-word shapes, through the context path and the no-allocation entry
point, and the decomposition rule."""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import assert_parity, compare_forces, force_errors, load_dem

pytestmark = pytest.mark.gpu

PRECISIONS = [0, 1, 2]
PNAMES = {0: "fp64", 1: "fp32", 2: "fp32c"}


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _cluster(shapes, ids, box, seed):
    rng = np.random.default_rng(seed)
    return W.contact_cluster(shapes, np.asarray(ids, np.int32), box, rng)


SYSTEMS = {
    "icospheres": lambda: _cluster([W.icosphere(0.7, 0.12)], np.zeros(90), [12.0] * 3, 31),
    "icospheres_mixed": lambda: _cluster([W.icosphere(0.7, 0.12), W.cube(0.9, 0.12), W.sphere(0.2)],
                                         np.arange(120) % 3, [12.0] * 3, 32),
    "polygon100": lambda: _cluster([W.polygon(100, 0.8, 0.1), W.square(1.0, 0.1)], np.arange(150) % 2,
                                   [36.0, 36.0], 33),
}
_cache = {}


def system(name):
    if name not in _cache:
        _cache[name] = SYSTEMS[name]()
    return _cache[name]


@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_wide_shape_parity(dem, name, precision):
    s = system(name)
    errs, ref, _ = compare_forces(dem, s, precision)
    assert ref["counts"][0, 2] > 0, "input must have contacts"
    assert_parity(errs, precision, f"wide/{name}/{PNAMES[precision]}")


def test_wide_shapes_run_thread(dem):
    """Only THREAD takes two-level masks: other decompositions are refused,
    and the autotuner times THREAD alone."""
    s = system("icospheres")
    with dem.DEM(s, dem.DEM_FP32_COMP) as d:
        assert d.get_param("decomp") == dem.DEM_DECOMP_THREAD
        for dec in (dem.DEM_DECOMP_WARP, dem.DEM_DECOMP_STAGED, dem.DEM_DECOMP_SPLIT):
            with pytest.raises(dem.DemError) as ei:
                d.set_param("decomp", dec)
            assert ei.value.code == dem.DEM_ERR_ARG
        dem.dem_autotune(d.ctx)
        assert d.get_param("decomp") == dem.DEM_DECOMP_THREAD
        assert d.get_param("autotune_ms_0") > 0 and d.get_param("autotune_ms_4") == -1
        d.step(20, 1e-3, dem.DEM_NVT)
        U, K, H = d.energy()
        assert np.isfinite(H).all()


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "fp32c"])
def test_wide_shape_trajectory(dem, precision):
    """Ten NVE steps of the icosphere cluster against the oracle's."""
    import oracle
    s = system("icospheres")
    ref, _ = oracle.run(s, 10, 1e-3, ensemble="nve")
    with dem.DEM(s, precision) as d:
        d.step(10, 1e-3, dem.DEM_NVE)
        st = d.state()
    dx = st["pos"] - ref["pos"]
    dx -= s.box[0] * np.round(dx / s.box[0])
    assert np.abs(dx).max() < (1e-9 if precision == 0 else 1e-6)


def test_wide_shape_noalloc(dem):
    import oracle
    import torch
    s = system("icospheres_mixed")
    ref = oracle.forces(s)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    f = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    e = torch.zeros((s.n,), dtype=torch.float64, device="cuda")
    dem.dem_forces_noalloc(s.shapes, s.epsilon, s.sigma, s.box[0], dev(s.shape_id, torch.int32),
                           dev(s.pos, torch.float64), dev(s.orient, torch.float64), 2, f, t, e)
    torch.cuda.synchronize()
    W6 = np.stack([[v[0, 0], 0.5 * (v[0, 1] + v[1, 0]), 0.5 * (v[0, 2] + v[2, 0]), v[1, 1],
                    0.5 * (v[1, 2] + v[2, 1]), v[2, 2]] for v in ref["virial"]])
    out = dict(force=f.cpu().numpy(), torque=t.cpu().numpy(), energy=e.cpu().numpy(),
               U=np.array([e.sum().item()]), W=W6, counts=None)
    assert_parity(force_errors(s, ref, out), 2, "wide/noalloc")
