"""Pins of the oracle's integrator: velocity Verlet with the symmetric
body-axis free-rotor splitting (Section "Energy Conservation": a second-
order integrator with dE/<E> ~ dt^2) and the Nose-Hoover thermostat on
translational and rotational degrees of freedom (Section "Assembly").

Pins: exact free flight; exact spin about a principal axis; exact
conservation of the world-frame angular momentum of a free asymmetric top;
time reversibility; the dt^2 scaling of the NVE energy error; conservation of
the NVT extended energy and its dt^2 scaling; thermalisation towards
equipartition.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.helpers import axis_angle_quat, copy_system, open_cluster, quat_mul, rotmat


def _single(shape, q, L_world, box=50.0):
    return W.System(3, [shape], np.zeros(1, np.int32), np.full((1, 3), box / 2),
                    np.array([q], float), np.zeros((1, 3)), np.array([L_world], float),
                    np.full((1, 3), box), np.array([1], np.int32), 1.0, 0.0)


def test_free_flight_exact(oracle_mod):
    rng = np.random.default_rng(0)
    n, L = 8, 200.0
    sh = W.cube(1.0, 0.15)
    pos = W.sc_sites([2, 2, 2], [L / 2] * 3)
    s = W.System(3, [sh], np.zeros(n, np.int32), pos, W.random_quaternions(rng, n),
                 rng.normal(size=(n, 3)), np.zeros((n, 3)), np.full((1, 3), L),
                 np.array([n], np.int32), 1.0, 0.0)
    st, _ = oracle_mod.run(s, 250, 0.01)
    expect = np.mod(pos + 2.5 * s.vel, L)
    np.testing.assert_allclose(st["pos"], expect, atol=1e-10)
    np.testing.assert_array_equal(st["vel"], s.vel)


def test_principal_axis_spin_exact(oracle_mod):
    sh = W.triangular_prism(1.0, 1.0, 0.15)
    q0 = axis_angle_quat([1, 2, 3], 0.7)
    Lz = 1.3
    Iz = sh["inertia"][2]
    s = _single(sh, q0, rotmat(q0) @ np.array([0, 0, Lz]))
    n, dt = 400, 0.005
    st, tr = oracle_mod.run(s, n, dt)
    expect = quat_mul(q0, axis_angle_quat([0, 0, 1], Lz / Iz * n * dt))
    got = st["orient"][0]
    assert min(np.abs(got - expect).max(), np.abs(got + expect).max()) < 1e-10
    np.testing.assert_allclose(tr[0, :, 1], 0.5 * Lz * Lz / Iz, rtol=1e-12)


def test_free_asymmetric_top(oracle_mod):
    sh = W.triangular_prism(1.0, 2.0, 0.15)        # I_x = I_y != I_z
    sh["inertia"] = np.array([0.2, 0.35, 0.1])      # make it fully asymmetric
    q0 = axis_angle_quat([0.2, -1, 0.4], 2.0)
    Lw = np.array([0.4, -0.9, 0.6])
    s = _single(sh, q0, Lw)
    st, tr = oracle_mod.run(s, 2000, 0.002)
    np.testing.assert_allclose(st["angmom"][0], Lw, atol=1e-12)
    assert abs(np.linalg.norm(st["orient"][0]) - 1) < 1e-14
    Kr = tr[0, :, 1]
    assert np.ptp(Kr) / Kr.mean() < 1e-4            # bounded O(dt^2) error of a splitting


def _cubes(seed=3, n=16):
    s = open_cluster([W.cube(1.0, 0.15)], np.zeros(n, np.int32), seed, gap=(0.95, 1.1),
                     gap_min=0.9)
    return s


def test_time_reversibility(oracle_mod):
    s = _cubes()
    st, _ = oracle_mod.run(s, 150, 0.002)
    back = copy_system(s, pos=st["pos"], orient=st["orient"], vel=-st["vel"],
                       angmom=-st["angmom"])
    st2, _ = oracle_mod.run(back, 150, 0.002)
    np.testing.assert_allclose(st2["pos"], s.pos, atol=1e-9)
    np.testing.assert_allclose(st2["vel"], -s.vel, atol=1e-8)
    qd = np.minimum(np.abs(st2["orient"] - s.orient).max(1),
                    np.abs(st2["orient"] + s.orient).max(1))
    assert qd.max() < 1e-9


def _herr(oracle_mod, s, dt, T, ens, **kw):
    n = int(round(T / dt))
    _, tr = oracle_mod.run(s, n, dt, ensemble=ens, **kw)
    H = tr[0, :, 3]
    o = oracle_mod.forces(s)
    K0 = 0.5 * (s.vel ** 2).sum() + 0.5 * sum(
        (rotmat(q).T @ L) @ ((rotmat(q).T @ L) / s.shapes[0]["inertia"])
        for q, L in zip(s.orient, s.angmom))
    H0 = K0 + o["U"][0]
    return np.abs(H - H0).max(), tr


@pytest.mark.parametrize("ens", ["nve", "nvt"])
def test_energy_error_scales_dt2(oracle_mod, ens):
    s = _cubes(seed=4, n=12)
    e1, tr = _herr(oracle_mod, s, 0.002, 0.2, ens, kT=1.0, tau=0.5)
    e2, _ = _herr(oracle_mod, s, 0.001, 0.2, ens, kT=1.0, tau=0.5)
    assert tr[0, :, 2].max() > 0.5, "the run must have interactions"
    assert 2.8 < e1 / e2 < 5.5, (e1, e2)


def test_nvt_thermalises(oracle_mod):
    s = _cubes(seed=6, n=16)
    s.vel[:] = 0.0
    s.angmom[:] = 0.0
    g = 3 * (s.n - 1) + 3 * s.n
    _, tr = oracle_mod.run(s, 3000, 0.002, ensemble="nvt", kT=1.0, tau=0.2)
    K = tr[0, :, 0] + tr[0, :, 1]
    assert K[1500:].mean() == pytest.approx(0.5 * g * 1.0, rel=0.35)
    H = tr[0, :, 3]
    assert np.ptp(H[100:]) < 0.02 * K[1500:].mean()


@pytest.mark.parametrize("name", ["dented", "lshapes"])
def test_energy_error_scales_dt2_concave(oracle_mod, name):
    """Concave shapes with disks / spheres nested in their notches and dents
    (Section "Model"): the spread of the conserved energy over a fixed time
    falls as dt^2 (Section "Energy Conservation": a second-order integrator)."""
    from tests.helpers import dent_points, nest_guests, notch_points
    if name == "dented":
        D = W.dented_cube(1.0, 0.6, 0.12)
        s = nest_guests(open_cluster([D], np.zeros(8, np.int32), 41), range(0, 8, 2),
                        W.sphere(0.15, 0.009), dent_points(D, 0.27), 41)
    else:
        L = W.l_shape2d(0.6, 0.12)
        s = nest_guests(open_cluster([L], np.zeros(10, np.int32), 42), range(0, 10, 2),
                        W.disk(0.15, 0.01), notch_points(L, 0.27), 42)
    spread = []
    for dt in (0.001, 0.0005):
        _, tr = oracle_mod.run(s, int(round(0.2 / dt)), dt, ensemble="nve")
        assert tr[0, :, 2].max() > 0.5, "the run must have interactions"
        spread.append(np.ptp(tr[0, :, 3]))
    assert 2.8 < spread[0] / spread[1] < 5.5, spread
