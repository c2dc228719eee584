"""dem_forces_noalloc: forces for callers that cannot call cudaMalloc.

Such callers (a framework whose pool allocator owns the device memory, a
process at its device-memory limit, a real-time loop that must not take the
synchronisation cudaMalloc / cudaFree can cause) get the forces of one
system from an entry point whose scratch is a static device array of the
library.  This test calls it through the C ABI, twice in a row on the same
inputs, and compares both results with the context path (dem_create,
dem_set_state, dem_get_forces) within the FP32 force tolerance of the other
GPU tests (tests/gpu_common.py), and checks that a size beyond the static
limit is refused.  It builds its own inputs, so it passes alone in a fresh
process and after the other tests.  The file name makes pytest collect it
last.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import TOL, load_dem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _system():
    rng = np.random.default_rng(77)
    return W.contact_cluster([W.cube(1.0, 0.15), W.tetrahedron(1.0, 0.12)],
                             np.arange(300) % 2, [13.0, 13.0, 13.0], rng)


@pytest.mark.parametrize("precision", [2, 0], ids=["fp32c", "fp64"])
def test_noalloc_matches_context(dem, precision):
    import torch
    import oracle
    s = _system()
    ref = oracle.forces(s)
    assert ref["counts"][0, 2] > 0
    with dem.DEM(s, precision) as d:
        f_ctx, t_ctx = d.forces()
        e_ctx = d.particle_energy()
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    sid = dev(s.shape_id, torch.int32)
    pos, ori = dev(s.pos, torch.float64), dev(s.orient, torch.float64)
    stream = torch.cuda.current_stream().cuda_stream
    S = np.maximum(ref["fscale"], 1e-300)
    T = np.maximum(ref["tscale"], 1e-300)
    active = ref["fscale"] > 0
    for call in range(2):
        f = torch.full((s.n, 3), np.nan, dtype=torch.float64, device="cuda")
        t = torch.full((s.n, 3), np.nan, dtype=torch.float64, device="cuda")
        e = torch.full((s.n,), np.nan, dtype=torch.float64, device="cuda")
        dem.dem_forces_noalloc(s.shapes, s.epsilon, s.sigma, s.box[0], sid, pos, ori,
                               precision, f, t, e, stream)
        torch.cuda.synchronize()
        f, t, e = f.cpu().numpy(), t.cpu().numpy(), e.cpu().numpy()
        errF = np.linalg.norm(f - f_ctx, axis=1)[active] / S[active]
        errT = np.linalg.norm(t - t_ctx, axis=1)[active] / T[active]
        assert errF.max() <= TOL[precision], (call, errF.max())
        assert errT.max() <= TOL[precision], (call, errT.max())
        assert np.all(f[~active] == 0.0) and np.all(t[~active] == 0.0)
        assert np.abs(e - e_ctx).max() <= TOL[precision] * (np.abs(e_ctx).max() + 1.0)


def test_noalloc_rejects_oversize(dem):
    import torch
    n = dem.DEM_NOALLOC_MAX_N + 1
    sh = W.sphere(0.3)
    z = lambda shape, dt: torch.zeros(shape, dtype=dt, device="cuda")
    with pytest.raises(dem.DemError) as ei:
        dem.dem_forces_noalloc([sh], 1.0, 0.0, [1000.0] * 3, z((n,), torch.int32),
                               z((n, 3), torch.float64), z((n, 4), torch.float64), 2,
                               z((n, 3), torch.float64), z((n, 3), torch.float64))
    assert ei.value.code == dem.DEM_ERR_ARG
