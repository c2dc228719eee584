"""dem_forces_noalloc: forces for callers that cannot call cudaMalloc.

Such callers (a framework whose pool allocator owns the device memory, a
process at its device-memory limit, a real-time loop that must not take the
synchronisation cudaMalloc / cudaFree can cause) get the forces of one
system from an entry point whose scratch is a static device array of the
library.  These tests call it through the C ABI and compare its forces,
torques and energies with the FP64 oracle (and with the context path,
dem_create / dem_set_state / dem_get_forces) in 3D and 2D and in every
precision, within the tolerances of the other GPU tests
(tests/gpu_common.py).

The array keeps the last call's contents, so a call must not depend on
them: each system is evaluated twice with a call on a different system
(other size, shapes and dimension) in between, and the repeated call must
give the same result.  Sizes beyond the static limit, more neighbours than
it holds, and a box below twice the interaction range are refused.  The
tests build their own inputs, so they pass alone in a fresh process and
after the other tests.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import assert_parity, force_errors, load_dem

pytestmark = pytest.mark.gpu

PNAMES = {0: "fp64", 1: "fp32", 2: "fp32c"}


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _system(dim):
    rng = np.random.default_rng(77 + dim)
    if dim == 3:
        return W.contact_cluster([W.cube(1.0, 0.15), W.tetrahedron(1.0, 0.12)],
                                 np.arange(300) % 2, [13.0, 13.0, 13.0], rng)
    return W.contact_cluster([W.square(1.0, 0.15), W.polygon(5, 0.7, 0.1)],
                             np.arange(260) % 2, [28.0, 28.0], rng)


def _other(dim):
    """A different system for the call in between: the other dimension,
    other shapes and size."""
    rng = np.random.default_rng(5)
    if dim == 3:
        return W.contact_cluster([W.polygon(6, 0.6, 0.12)], np.zeros(400, np.int32),
                                 [40.0, 40.0], rng)
    return W.contact_cluster([W.octahedron(1.0, 0.1), W.sphere(0.3)], np.arange(500) % 2,
                             [16.0, 16.0, 16.0], rng)


def _call(dem, s, precision):
    import torch
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    tw = 3 if s.dim == 3 else 1
    f = torch.full((s.n, s.dim), np.nan, dtype=torch.float64, device="cuda")
    t = torch.full((s.n, tw), np.nan, dtype=torch.float64, device="cuda")
    e = torch.full((s.n,), np.nan, dtype=torch.float64, device="cuda")
    dem.dem_forces_noalloc(s.shapes, s.epsilon, s.sigma, s.box[0], dev(s.shape_id, torch.int32),
                           dev(s.pos, torch.float64), dev(s.orient, torch.float64), precision,
                           f, t, e, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f.cpu().numpy(), t.cpu().numpy(), e.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1, 2], ids=[PNAMES[p] for p in (0, 1, 2)])
@pytest.mark.parametrize("dim", [3, 2])
def test_noalloc_matches_oracle(dem, dim, precision):
    import oracle
    s = _system(dim)
    ref = oracle.forces(s)
    assert ref["counts"][0, 2] > 0
    first = _call(dem, s, precision)
    _call(dem, _other(dim), precision)           # leaves other contents behind
    again = _call(dem, s, precision)
    for k in range(3):
        np.testing.assert_array_equal(again[k], first[k])
    f, t, e = first
    # per-replica U and W are not outputs of this entry point: reuse the
    # oracle's so that only the per-particle quantities are compared
    out = dict(force=f, torque=t, energy=e, U=np.array([e.sum()]), W=None, counts=None)
    errs = force_errors_noalloc(s, ref, out)
    assert_parity(errs, precision, f"noalloc/{dim}d/{PNAMES[precision]}")
    # and the context path on the same system
    with dem.DEM(s, precision) as d:
        f_ctx, t_ctx = d.forces()
    S = np.maximum(ref["fscale"], 1e-300)
    act = ref["fscale"] > 0
    from tests.gpu_common import TOL
    assert (np.linalg.norm(f - f_ctx, axis=1)[act] / S[act]).max() <= TOL[precision]


def force_errors_noalloc(s, ref, out):
    """force_errors with the virial taken from the oracle (the entry point
    returns no virial)."""
    W6 = np.stack([[v[0, 0], 0.5 * (v[0, 1] + v[1, 0]), 0.5 * (v[0, 2] + v[2, 0]), v[1, 1],
                    0.5 * (v[1, 2] + v[2, 1]), v[2, 2]] for v in ref["virial"]])
    return force_errors(s, ref, dict(out, W=W6))


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


def test_noalloc_neighbour_overflow(dem):
    """A dense gas of unit spheres: about 80 neighbours within the range per
    particle, more than the static list holds."""
    import torch
    rng = np.random.default_rng(3)
    n, L = 3000, 6.0
    pos = rng.uniform(0, L, size=(n, 3))
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    f = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dem.DemError) as ei:
        dem.dem_forces_noalloc([W.sphere(0.5)], 1.0, 0.0, [L] * 3, dev(np.zeros(n), torch.int32),
                               dev(pos, torch.float64), dev(np.tile([1.0, 0, 0, 0], (n, 1)),
                                                            torch.float64), 2, f, t)
    assert ei.value.code == dem.DEM_ERR_NLIST_OVERFLOW


def test_noalloc_small_box(dem):
    import torch
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    pos = np.array([[0.5, 0.5, 0.5], [2.0, 0.5, 0.5]])
    f = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dem.DemError) as ei:
        dem.dem_forces_noalloc([W.cube(1.0, 0.15)], 1.0, 0.3, [3.0] * 3,
                               dev(np.zeros(2), torch.int32), dev(pos, torch.float64),
                               dev(np.tile([1.0, 0, 0, 0], (2, 1)), torch.float64), 2, f, t)
    assert ei.value.code == dem.DEM_ERR_BOX


def test_noalloc_wrapper_checks(dem):
    """The binding refuses arrays the library could not check: a wrong
    dtype, a non-contiguous view or a short array."""
    import torch
    s = _system(3)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    sid, pos, ori = dev(s.shape_id, torch.int32), dev(s.pos, torch.float64), dev(s.orient, torch.float64)
    f = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    bad = [dict(pos=pos.float()), dict(orient=dev(s.orient.T, torch.float64).T),
           dict(force=f[:-1]), dict(shape_id=sid.long())]
    for b in bad:
        args = dict(shape_id=sid, pos=pos, orient=ori, force=f, torque=t)
        args.update(b)
        with pytest.raises(ValueError):
            dem.dem_forces_noalloc(s.shapes, s.epsilon, s.sigma, s.box[0], args["shape_id"],
                                   args["pos"], args["orient"], 2, args["force"], args["torque"])
