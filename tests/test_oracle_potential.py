"""Pins of the oracle's pair potential (Eq. LJ, Eq. WCA) and of the sphere
limit (spheres interact through the central WCA, Section "Performance").

Each check is a fact fixed by the mathematics, not a retyped formula:
U(sigma) = eps (LJ vanishes at sigma, the shift adds eps), U -> 0 and F -> 0
at r_cut = 2^(1/6) sigma (the LJ minimum), a hand-evaluated value, the
scaling law in eps and sigma, and F = -dU/dr by finite differences.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.helpers import two_body


@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (1.0, 0.3), (2.5, 0.2)])
def test_wca_closed_form_points(oracle_mod, eps, sigma):
    u, f = oracle_mod.wca(sigma, eps, sigma)
    assert u == pytest.approx(eps, rel=1e-14)                    # U(sigma) = eps
    assert f == pytest.approx(24 * eps / sigma, rel=1e-14)       # -U'(sigma) = 24 eps/sigma
    # (sigma/r)^6 = 2  ->  U_LJ = 4 eps (4 - 2) = 8 eps, plus the shift eps
    r = sigma * 0.5 ** (1 / 6)
    assert oracle_mod.wca(r, eps, sigma)[0] == pytest.approx(9 * eps, rel=1e-13)
    rc = 2 ** (1 / 6) * sigma
    u, f = oracle_mod.wca(rc * (1 - 1e-9), eps, sigma)
    assert abs(u) < 1e-14 * eps * 1e3 and abs(f) < 1e-6 * eps / sigma
    assert oracle_mod.wca(rc, eps, sigma) == (0.0, 0.0)
    assert oracle_mod.wca(1.5 * rc, eps, sigma) == (0.0, 0.0)


def test_wca_scaling_and_derivative(oracle_mod):
    rs = np.linspace(0.85, 1.12, 41)
    for eps, sigma in [(1.0, 0.3), (3.0, 0.17)]:
        for x in rs:
            u, f = oracle_mod.wca(x * sigma, eps, sigma)
            u1, f1 = oracle_mod.wca(x, 1.0, 1.0)
            assert u == pytest.approx(eps * u1, rel=1e-12, abs=1e-15)
            assert f == pytest.approx(eps / sigma * f1, rel=1e-12, abs=1e-12)
            h = 1e-6 * sigma
            if x * sigma + h < 2 ** (1 / 6) * sigma:
                fd = -(oracle_mod.wca(x * sigma + h, eps, sigma)[0]
                       - oracle_mod.wca(x * sigma - h, eps, sigma)[0]) / (2 * h)
                assert fd == pytest.approx(f, rel=1e-6)


def test_wca_monotone_repulsive(oracle_mod):
    rs = np.linspace(0.8, 2 ** (1 / 6) - 1e-6, 200)
    us = np.array([oracle_mod.wca(r, 1.0, 1.0)[0] for r in rs])
    fs = np.array([oracle_mod.wca(r, 1.0, 1.0)[1] for r in rs])
    assert np.all(np.diff(us) < 0) and np.all(us > 0) and np.all(fs > 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_sphere_limit_pair(oracle_mod, dim):
    sh = W.sphere(0.15) if dim == 3 else W.disk(0.15)
    rng = np.random.default_rng(7)
    for r in np.linspace(0.26, 0.34, 9):
        u = rng.normal(size=dim)
        u /= np.linalg.norm(u)
        s = two_body(sh, sh, r * u)
        dv = s.pos[1] - s.pos[0]          # the separation as stored
        r = np.linalg.norm(dv)
        u = dv / r
        o = oracle_mod.forces(s)
        ue, fe = oracle_mod.wca(r, 1.0, 0.3)
        assert o["U"][0] == pytest.approx(ue, rel=1e-13, abs=1e-15)
        # central force along the centre line, equal and opposite, no torque
        np.testing.assert_allclose(o["force"][0], -fe * u, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(o["force"][1], fe * u, rtol=1e-12, atol=1e-12)
        assert np.abs(o["torque"]).max() < 1e-12
        assert o["counts"][0, 2] == (1 if r < 2 ** (1 / 6) * 0.3 else 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_sphere_limit_gas(oracle_mod, dim):
    """A periodic gas of spheres: the total is the central WCA pair sum."""
    rng = np.random.default_rng(11 + dim)
    n, L = 120, 6.0 if dim == 3 else 10.0
    sh = W.sphere(0.25) if dim == 3 else W.disk(0.25)
    pos = rng.random((n, dim)) * L
    s = W.System(dim, [sh], np.zeros(n, np.int32), pos,
                 np.tile([1.0, 0, 0, 0], (n, 1)) if dim == 3 else np.zeros((n, 1)),
                 np.zeros((n, dim)), np.zeros((n, 3 if dim == 3 else 1)),
                 np.full((1, dim), L), np.array([n], np.int32), 1.0, 0.0)
    o = oracle_mod.forces(s)
    tot, fsum = 0.0, np.zeros((n, dim))
    for i in range(n):
        for j in range(i + 1, n):
            d = pos[j] - pos[i]
            d -= L * np.round(d / L)
            r = np.linalg.norm(d)
            u, f = oracle_mod.wca(r, 1.0, 0.5)
            tot += u
            fsum[i] -= f * d / r
            fsum[j] += f * d / r
    assert o["U"][0] == pytest.approx(tot, rel=1e-12)
    np.testing.assert_allclose(o["force"], fsum, rtol=1e-10, atol=1e-9)
