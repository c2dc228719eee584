"""The timed CPU baseline's form of the oracle (cell-list pair search,
OpenMP over particles) against the plain all-pairs, single-thread oracle:
the same pairs and terms, so the same forces, torques, energies, virial and
counts up to the order of the sums; the same trajectories over a few
steps."""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W


def _systems():
    rng = np.random.default_rng(9)
    yield "cubes", W.contact_cluster([W.cube(1.0, 0.15)], np.zeros(150, np.int32), [12.0] * 3,
                                     rng, sigma=0.3)
    yield "mixed", W.contact_cluster([W.tetrahedron(1.0, 0.1), W.sphere(0.3), W.octahedron(0.9, 0.12)],
                                     np.arange(160) % 3, [11.0] * 3, rng)
    yield "squares", W.contact_cluster([W.square(1.0, 0.15)], np.zeros(200, np.int32), [28.0] * 2,
                                       rng, sigma=0.3)
    # a box with fewer than three cells per axis: every pair
    yield "small_box", W.contact_cluster([W.cube(1.0, 0.15)], np.zeros(10, np.int32), [6.0] * 3,
                                         rng, sigma=0.3)


@pytest.mark.parametrize("threads,cells", [(1, True), (4, False), (4, True)])
def test_parallel_forces_match_plain(oracle_mod, threads, cells):
    for name, s in _systems():
        oracle_mod.set_parallel(1, False)
        ref = oracle_mod.forces(s, scales=False)
        try:
            oracle_mod.set_parallel(threads, cells)
            # scales=False: the plain evaluation is used whenever scales or
            # flags are requested
            got = oracle_mod.forces(s, scales=False)
        finally:
            oracle_mod.set_parallel(1, False)
        assert got["counts"].tolist() == ref["counts"].tolist(), name
        sc = np.abs(ref["force"]).max()
        np.testing.assert_allclose(got["force"], ref["force"], rtol=0, atol=1e-12 * sc, err_msg=name)
        np.testing.assert_allclose(got["torque"], ref["torque"], rtol=0,
                                   atol=1e-12 * np.abs(ref["torque"]).max(), err_msg=name)
        np.testing.assert_allclose(got["energy"], ref["energy"], rtol=1e-12, atol=1e-12, err_msg=name)
        np.testing.assert_allclose(got["virial"], ref["virial"], rtol=1e-11,
                                   atol=1e-12 * np.abs(ref["virial"]).max(), err_msg=name)


def test_parallel_run_matches_plain(oracle_mod):
    s = next(_systems())[1]
    a, _ = oracle_mod.run(s, 20, 1e-3, ensemble="nvt")
    try:
        oracle_mod.set_parallel(4, True)
        b, _ = oracle_mod.run(s, 20, 1e-3, ensemble="nvt")
    finally:
        oracle_mod.set_parallel(1, False)
    np.testing.assert_allclose(b["pos"], a["pos"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(b["vel"], a["vel"], rtol=0, atol=1e-9)
