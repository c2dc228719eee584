"""GPU parity of the method's own edge cases (Section "Model"): the
parallel-edge rule, exactly parallel and collinear edges, the face-to-face
overcounting example, vertices projecting exactly onto a face's boundary,
and aligned lattices in periodic boxes where every edge pair is exactly
parallel or perpendicular.  Every precision and every pair-kernel
decomposition is compared element by element with the FP64 oracle through
the C ABI (tolerances: tests/gpu_common.py).

The constructions (tests/helpers.py) are pinned on the CPU in
tests/test_oracle_edge_cases.py: the in-band ridge pairs reach the rule
(their torques change when it is switched off), the out-of-band ones do not,
and the face-to-face pair has the 56 terms of tests/golden/overcount.txt.
None of these inputs has a squared sine within a decade of the band's
threshold, so no particle is excluded: the tests require zero flagged.
"""
import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W
from tests.gpu_common import assert_parity, compare_forces, load_dem
from tests.helpers import (aligned_lattice, collinear_ridges, face_to_face, ridge_pair,
                           square_pairs_2d, swap_pair, vertex_over_face_edge)

pytestmark = pytest.mark.gpu

PRECISIONS = [0, 1, 2]
PNAMES = {0: "fp64", 1: "fp32", 2: "fp32c"}
DECOMPS = {"thread": 1, "warp": 2, "staged": 3, "split": 4}

# squared sines of the ridge pairs: exactly parallel, two inside the band
# (threshold 1e-6), one far outside it
SIN2 = [0.0, 1e-8, 5e-8, 1e-4]


@pytest.fixture(scope="module")
def dem():
    return load_dem()


def _edge_cases_3d():
    reps = []
    for s2 in SIN2:
        reps.append(ridge_pair(s2, 0.3, 0.28))       # overlapping projections
        reps.append(ridge_pair(s2, 1.2, 0.2))        # no overlap: endpoint pairs
    # the in-band pairs in the other order: the other ridge is the reference
    reps.append(swap_pair(ridge_pair(5e-8, 0.3, 0.28)))
    reps.append(swap_pair(ridge_pair(1e-8, 0.3, 0.28)))
    for gap in (0.27, 0.30, 0.32, 0.335):
        reps.append(face_to_face(gap))
    reps.append(face_to_face(0.29, lateral=(0.3, 0.45)))
    reps.append(collinear_ridges(0.28))
    reps.append(vertex_over_face_edge(0.28))
    reps.append(vertex_over_face_edge(0.28, corner=True))
    return W.merge(reps, "edge_cases_3d")


SYSTEMS = {
    "edge_cases_3d": _edge_cases_3d,
    "aligned_cubes": lambda: aligned_lattice(3, 6, 0.31, 0.015, 1),
    "aligned_squares": lambda: aligned_lattice(2, 12, 0.31, 0.015, 2),
    "square_pairs": lambda: square_pairs_2d(0.3),
}
_cache = {}


def system(name):
    if name not in _cache:
        _cache[name] = SYSTEMS[name]()
    return _cache[name]


@pytest.mark.parametrize("decomp", list(DECOMPS))
@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_edge_case_parity(dem, name, precision, decomp):
    s = system(name)
    errs, ref, out = compare_forces(dem, s, precision, decomp=DECOMPS[decomp])
    assert ref["counts"][:, 2].min() > 0, "every replica must have contacts"
    assert errs["flagged"] == 0
    assert_parity(errs, precision, f"edge/{name}/{PNAMES[precision]}/{decomp}", flagged_max=0.0)
    if precision == 0:     # per-replica energies, replica by replica
        np.testing.assert_allclose(out["U"], ref["U"], rtol=1e-12)


@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
def test_face_to_face_terms_on_gpu(dem, precision):
    """The worked example of Section "Model" on the GPU: 56 terms at the face
    gap, U = 56 U(gap), force along the face normal, no torque.  Errors are
    measured against the terms' scale 56 (|f| + sigma |f'|), as in
    tests/gpu_common.py."""
    import oracle
    from tests.gpu_common import TOL
    sig = 0.3
    for gap in (0.27, 0.30, 0.32, 0.335):
        s = face_to_face(gap, sigma=sig)
        u1, f1 = oracle.wca(gap, 1.0, sig)
        h = 1e-7
        df = (oracle.wca(gap + h, 1.0, sig)[1] - oracle.wca(gap - h, 1.0, sig)[1]) / (2 * h)
        scale = 56 * (abs(f1) + sig * abs(df))
        with dem.DEM(s, precision, decomp=4) as d:
            f, t = d.forces()
            U, _, _ = d.energy()
            cnt = d.counters()
        tol = TOL[precision]
        assert cnt[2] == 2 * 56, (gap, cnt[2])
        assert abs(U[0] - 56 * u1) <= tol * sig * scale
        assert np.abs(f[1] - [0, 0, 56 * f1]).max() <= tol * scale
        assert np.abs(f[0] + f[1]).max() <= tol * scale
        assert np.abs(t).max() <= tol * scale


@pytest.mark.parametrize("precision", PRECISIONS, ids=[PNAMES[p] for p in PRECISIONS])
def test_parallel_rule_switch(dem, precision):
    """A ridge pair inside the band (squared sine 1e-8) gives the rule's
    torque with par_eps = 1e-6 and the ordinary nearest points' torque with
    par_eps = 0, each matching the oracle run with the same threshold.  The
    ordinary solution of nearly parallel edges divides by the squared sine,
    which FP32 cannot resolve at 1e-8 (the reason for the rule): with
    par_eps = 0 only FP64 is compared."""
    import oracle
    s = ridge_pair(1e-8, 0.3, 0.28)
    tq = {}
    for pe in ((1e-6, 0.0) if precision == 0 else (1e-6,)):
        ref = oracle.forces(s, par_eps=pe)
        with dem.DEM(s, precision, decomp=4, par_eps=pe) as d:
            f, t = d.forces()
        scale = np.abs(ref["torque"]).max()
        np.testing.assert_allclose(t, ref["torque"], atol=(1e-10 if precision == 0 else 1e-4) * scale)
        tq[pe] = t
    # the two readings differ by far more than the tolerance
    if precision == 0:
        assert np.abs(tq[1e-6] - tq[0.0]).max() > 0.05 * np.abs(tq[0.0]).max()
