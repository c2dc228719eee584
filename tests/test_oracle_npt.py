"""Pins of the oracle's isotropic barostat (ensemble "npt": the MTK equations
integrated as in Tuckerman et al. 2006, cited by Section "Assembly" for the
NPT runs; the paper gives no formulas, so the scheme is the reading stated in
oracle/dem_oracle.c).

Pins: the conserved quantity K + U + p_e^2/2W + P V + (g+1) kT (tau^2 xi^2/2 +
eta) holds with an error that scales as dt^2 (a wrong factor or sign in any
sub-step breaks it); the scheme is time reversible (negating v, L, p_e and
xi retraces the path, box included); the volume falls under a high pressure
and grows when the applied pressure is zero; without a barostat
(ensemble "nvt") the box never changes.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.helpers import copy_system, rotmat


def _dense(seed=11, n=24, box=7.0):
    rng = np.random.default_rng(seed)
    return W.contact_cluster([W.cube(1.0, 0.15)], np.zeros(n, np.int32), [box] * 3, rng,
                             gap=(0.95, 1.1), gap_min=0.9, free=0.0)


def _h0(oracle_mod, s, P):
    o = oracle_mod.forces(s)
    K0 = 0.5 * (s.vel ** 2).sum() + 0.5 * sum(
        (rotmat(q).T @ L) @ ((rotmat(q).T @ L) / s.shapes[0]["inertia"])
        for q, L in zip(s.orient, s.angmom))
    return K0 + o["U"][0] + P * np.prod(s.box[0])


def _herr(oracle_mod, s, dt, T, P, tau_P):
    n = int(round(T / dt))
    st, tr = oracle_mod.run(s, n, dt, ensemble="npt", kT=1.0, tau=0.5, P=P, tau_P=tau_P)
    return np.abs(tr[0, :, 3] - _h0(oracle_mod, s, P)).max(), st, tr


def test_npt_conserved_quantity_scales_dt2(oracle_mod):
    s = _dense()
    e1, st, tr = _herr(oracle_mod, s, 0.002, 0.3, P=2.0, tau_P=0.3)
    e2, _, _ = _herr(oracle_mod, s, 0.001, 0.3, P=2.0, tau_P=0.3)
    assert tr[0, :, 2].max() > 0.5, "the run must have interactions"
    assert abs(tr[0, -1, 4] / np.prod(s.box[0]) - 1.0) > 1e-3, "the box must move"
    assert 2.8 < e1 / e2 < 5.5, (e1, e2)


def test_npt_time_reversible(oracle_mod):
    s = _dense(seed=12)
    st, _ = oracle_mod.run(s, 120, 0.002, ensemble="npt", kT=1.0, tau=0.5, P=2.0, tau_P=0.3)
    assert abs(np.prod(st["box"][0]) / np.prod(s.box[0]) - 1.0) > 1e-3
    th = st["thermo"].copy()
    th[:, 0] *= -1.0          # xi
    th[:, 2] *= -1.0          # p_e
    back = copy_system(s, pos=st["pos"], orient=st["orient"], vel=-st["vel"],
                       angmom=-st["angmom"], box=st["box"])
    st2, _ = oracle_mod.run(back, 120, 0.002, ensemble="npt", kT=1.0, tau=0.5, P=2.0,
                            tau_P=0.3, thermo=th)
    np.testing.assert_allclose(st2["box"], s.box, rtol=1e-11)
    d = st2["pos"] - s.pos
    d -= s.box[0] * np.round(d / s.box[0])
    assert np.abs(d).max() < 1e-8
    np.testing.assert_allclose(st2["vel"], -s.vel, atol=1e-7)
    assert np.abs(st2["thermo"][:, [0, 2]]).max() < 1e-9


@pytest.mark.parametrize("P,sign", [(0.5, -1), (0.0, 1)])
def test_npt_volume_follows_pressure(oracle_mod, P, sign):
    s = _dense(seed=13)
    _, tr = oracle_mod.run(s, 150, 0.002, ensemble="npt", kT=1.0, tau=0.5, P=P, tau_P=1.0)
    assert np.all(np.isfinite(tr))
    dv = tr[0, -1, 4] - np.prod(s.box[0])
    assert sign * dv > 0.01 * np.prod(s.box[0])


def test_nvt_keeps_the_box(oracle_mod):
    s = _dense(seed=14)
    st, tr = oracle_mod.run(s, 50, 0.002, ensemble="nvt", kT=1.0, tau=0.5, P=50.0, tau_P=0.2)
    np.testing.assert_array_equal(st["box"], s.box)
    assert np.all(tr[0, :, 4] == np.prod(s.box[0]))


@pytest.mark.parametrize("P", [1.0, 3.0])
def test_npt_mean_pressure_is_the_set_pressure(oracle_mod, P):
    """At equilibrium the barostat's equation dp_e/dt = alpha 2 K_trans +
    Tr W - d V P averages to zero, so the time average of the instantaneous
    pressure (alpha 2 K_trans + Tr W) / (d V) is the applied P.  A barostat
    that conserves its H but drives towards the wrong pressure (a missing or
    mis-signed virial, a wrong alpha or kinetic factor) fails this.  WCA
    spheres (64, a fluid near the set pressure), 4000 steps to equilibrate,
    then 400 samples 50 steps apart; the block-average scatter of the mean is
    about 0.5% of P."""
    import dataclasses
    rng = np.random.default_rng(3)
    a = 1.25
    pos = W.sc_sites([4] * 3, [a] * 3)
    n = len(pos)
    s = W._finish(rng, 3, [W.sphere(0.5)], np.zeros(n, np.int32), pos, np.full(3, 4 * a), [n],
                  1.0, orient=np.tile([1.0, 0, 0, 0], (n, 1)))
    kw = dict(ensemble="npt", kT=1.0, tau=0.5, P=P, tau_P=1.0)

    def advance(s, steps, th):
        st, _ = oracle_mod.run(s, steps, 0.005, thermo=th, **kw)
        return dataclasses.replace(s, pos=st["pos"], orient=st["orient"], vel=st["vel"],
                                   angmom=st["angmom"], box=st["box"]), st["thermo"]

    s, th = advance(s, 4000, None)
    alpha = 1.0 + 3.0 / (3.0 * (n - 1))
    p_inst = []
    for _ in range(400):
        s, th = advance(s, 50, th)
        kt = 0.5 * (s.vel ** 2).sum()
        vir = oracle_mod.forces(s, scales=False)["virial"][0]
        p_inst.append((alpha * 2.0 * kt + np.trace(vir)) / (3.0 * np.prod(s.box[0])))
    assert np.mean(p_inst) == pytest.approx(P, rel=0.03)
