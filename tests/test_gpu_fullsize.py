"""Parity at full size, in the launch configuration the bench times
(autotuned decomposition, one force evaluation of the whole workload):

* the batched workload (512 replicas, 551,213 particles), prepared as the
  bench prepares it (compressed on the GPU to the target densities, then
  equilibrated): every particle of 16 replicas spread over the batch against
  the oracle run on each of those replicas;
* the single 1,048,576-cube system (packing fraction 0.55), prepared as the
  bench prepares it (compressed on the GPU from the safe lattice start, then
  equilibrated): sampled particles against the oracle run on each one's
  neighbourhood (the particle and every particle that can reach it,
  unwrapped into an empty box, so that the oracle's force, torque and energy
  on that particle are exact), plus Newton's third law over the whole
  system.
"""
import numpy as np
import pytest

import oracle
from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import TOL, assert_parity, force_errors, load_dem

pytestmark = pytest.mark.gpu

SAMPLE_REPLICAS = [0, 1, 2, 63, 64, 65, 127, 200, 255, 256, 300, 383, 400, 451, 510, 511]


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _prepared(dem, s0, steps=3000, equil=300):
    """The workload's state after the bench's preparation."""
    import bench
    run = dict(dt=1e-3, ensemble="nvt", kT=1.0, tau=0.5)
    d = bench.prepare(dem, s0, run, dem.DEM_FP32_COMP, steps, equil)
    try:
        st = d.state()
    finally:
        d.close()
    return W.System(s0.dim, s0.shapes, s0.shape_id, st["pos"], st["orient"], st["vel"],
                    st["angmom"], st["box"], s0.replica_sizes, s0.epsilon, s0.sigma)


@pytest.fixture(scope="module")
def batched(dem):
    return _prepared(dem, W.config_batched())


def _gpu(dem, system, precision):
    with dem.DEM(system, precision) as d:
        dem.dem_autotune(d.ctx)
        f, t = d.forces()
        U, K, H = d.energy()
        return dict(force=f, torque=t, U=U, W=d.virial(), energy=d.particle_energy(),
                    decomp=int(d.get_param("decomp")))


@pytest.mark.parametrize("precision", [2, 0], ids=["fp32c", "fp64"])
def test_batched_full_size_sampled_replicas(dem, batched, precision):
    out = _gpu(dem, batched, precision)
    slices = batched.replica_slices()
    live = 0
    for k in SAMPLE_REPLICAS:
        sl = slices[k]
        rep = batched.replica(k)
        ref = oracle.forces(rep)
        live += int((ref["fscale"] > 0).sum())
        sub = dict(force=out["force"][sl], torque=out["torque"][sl], energy=out["energy"][sl],
                   U=out["U"][k:k + 1], W=out["W"][k:k + 1], counts=None)
        errs = force_errors(rep, ref, sub)
        assert_parity(errs, precision, f"fullsize batched/{k}/decomp{out['decomp']}")
    assert live > 1000, "the sample must have contacts"


def _local_oracle(system, i, reach):
    """Oracle force, torque, energy and scales of particle i from its
    neighbourhood (all j with |x_j - x_i| < reach, minimum image), unwrapped
    into an empty box."""
    L = system.box[0]
    d = system.pos - system.pos[i]
    d -= L * np.round(d / L)
    near = np.nonzero(np.linalg.norm(d, axis=1) < reach)[0]
    near = np.concatenate([[i], near[near != i]])
    big = 4.0 * reach + 10.0
    sub = W.System(3, system.shapes, system.shape_id[near], d[near] + big / 2,
                   system.orient[near], system.vel[near], system.angmom[near],
                   np.full((1, 3), big), np.array([len(near)], np.int32), system.epsilon,
                   system.sigma)
    return oracle.forces(sub), sub


def test_large_system_sampled_particles(dem):
    s = _prepared(dem, W.config_large())
    out = _gpu(dem, s, 2)
    f, t, e = out["force"], out["torque"], out["energy"]
    # Newton's third law over the whole system (FP32 terms, compensated sums)
    scale = np.abs(f).sum()
    assert scale > 0, "the state must have contacts"
    assert np.abs(f.sum(0)).max() < 1e-6 * scale
    # sampled particles against the oracle on their neighbourhoods
    rng = np.random.default_rng(7)
    sh = s.shapes[0]
    R = float(np.max(np.linalg.norm(sh["verts"], axis=1)))
    sig = s.sigma if s.sigma > 0 else 2 * sh["rounding"]
    reach = 2 * R + 2 ** (1 / 6) * sig + 0.1
    live = 0
    for i in rng.choice(s.n, size=48, replace=False):
        ref, sub = _local_oracle(s, int(i), reach)
        if ref["flags"][0] or ref["fscale"][0] == 0:
            assert np.all(f[i] == 0) or ref["flags"][0]
            continue
        live += 1
        errF = np.linalg.norm(f[i] - ref["force"][0]) / ref["fscale"][0]
        errT = np.linalg.norm(t[i] - ref["torque"][0]) / ref["tscale"][0]
        errU = abs(e[i] - ref["energy"][0]) / (sig * ref["fscale"][0])
        assert max(errF, errT, errU) < TOL[2], (int(i), errF, errT, errU)
    assert live >= 10, "the sample must have contacts"
