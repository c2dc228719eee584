"""CPU-side checks of the CUDA library: it builds, loads, exports every
symbol include/dem.h declares, and its host-only shape preprocessing
(dem_shape_info) gives the closed-form properties of the workload shapes.
No CUDA device is used."""
import os
import re

import numpy as np
import pytest

from paper_1607_02427_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dem():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_02427_gb300 import dem as d
    return d


def _declared():
    src = open(os.path.join(ROOT, "include", "dem.h")).read()
    return sorted(set(re.findall(r"\b(dem_[a-z_]+)\s*\(", src)) - {"dem_shape"})


def test_exports_match_header(dem):
    lib = dem.load()
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), f"libdem.so does not export {name}"
    assert sorted(dem.EXPORTS) == declared


def test_sm103a_only(dem):
    """The library is built for sm_103a: the build flags name it."""
    from paper_1607_02427_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


@pytest.mark.parametrize("name,mk,expect", [
    ("cube", lambda: W.cube(1.0, 0.15), [1 / 6, 1 / 6, 1 / 6]),
    ("tetrahedron", lambda: W.tetrahedron(1.0, 0.15), [1 / 20] * 3),
    ("octahedron", lambda: W.octahedron(1.0, 0.1), [1 / 5] * 3),
    ("prism", lambda: W.triangular_prism(1.0, 1.0, 0.15),
     [1 / 24 + 1 / 12, 1 / 24 + 1 / 12, 1 / 12]),
    ("icosahedron", lambda: W.icosahedron(1.0, 0.15), [((1 + 5 ** .5) / 2) ** 2 / 10] * 3),
])
def test_shape_info_3d(dem, name, mk, expect):
    sh = mk()
    sh = dict(sh, inertia=None)
    info = dem.dem_shape_info(sh)
    assert info[0] == pytest.approx(W.circumradius(sh), rel=1e-12)
    np.testing.assert_allclose(info[2:5], expect, rtol=1e-12)
    assert info[5] == pytest.approx(sh["inner_measure"], rel=1e-12)
    assert info[6] < 1e-12
    n_edges = {"cube": 12, "tetrahedron": 6, "octahedron": 12, "prism": 9, "icosahedron": 30}
    assert info[1] == n_edges[name]


def test_shape_info_2d(dem):
    sq = dict(W.square(1.0, 0.15), inertia=None)
    info = dem.dem_shape_info(sq)
    assert info[1] == 4 and info[2] == pytest.approx(1 / 6) and info[5] == pytest.approx(1.0)
    pent = dict(W.polygon(5, 0.7, 0.1), inertia=None)
    assert dem.dem_shape_info(pent)[2] == pytest.approx(W.polygon(5, 0.7, 0.1)["inertia"][0],
                                                        rel=1e-12)


def test_shape_info_concave(dem):
    """Concave shapes (Section "Model"): the library's derived mass
    properties equal the closed forms (L-shape: area 3 a^2, I_z = 11 a^2/18;
    dented cube: volume a^3 - a^2 h / 3, I_zz = (a^5/6 - a^4 h/30) / V)."""
    L = dict(W.l_shape2d(1.0, 0.15), inertia=None)
    info = dem.dem_shape_info(L)
    assert info[1] == 6
    assert info[2] == pytest.approx(11 / 18, rel=1e-12)
    assert info[5] == pytest.approx(3.0, rel=1e-12)
    a, h = 1.0, 0.5
    D = W.dented_cube(a, h, 0.15)
    info = dem.dem_shape_info(dict(D, inertia=None))
    V = a ** 3 - a * a * h / 3
    assert info[1] == 16
    assert info[5] == pytest.approx(V, rel=1e-12)
    assert info[4] == pytest.approx((a ** 5 / 6 - a ** 4 * h / 30) / V, rel=1e-12)
    np.testing.assert_allclose(info[2:5], D["inertia"], rtol=1e-12)
    assert info[6] < 1e-12


@pytest.mark.parametrize("bad", ["inward", "flipped_face", "open", "nonplanar", "nonconvex_face",
                                 "bowtie", "clockwise", "fold", "offcentre", "rounding"])
def test_shape_validation(dem, bad):
    sh = W.cube(1.0, 0.15)
    sh = dict(sh, inertia=None)
    if bad == "inward":
        sh["faces"] = [list(reversed(f)) for f in sh["faces"]]
    elif bad == "flipped_face":
        sh["faces"] = [list(reversed(f)) if k == 2 else f for k, f in enumerate(sh["faces"])]
    elif bad == "open":
        sh = dict(W.dented_cube(1.0, 0.5, 0.15))
        sh["faces"] = sh["faces"][:-1]
    elif bad == "nonplanar":
        sh["verts"] = sh["verts"].copy()
        sh["verts"][6, 2] += 0.05
        sh["inertia"] = [1 / 6] * 3
    elif bad == "nonconvex_face":
        # a dart-shaped top face: the nearest point on a face needs convex faces
        v = np.array([[-1, -1, 0], [1, -1, 0], [0, -0.2, 0], [-1, 1, 0], [0, 0, -1.0]])
        sh = dict(dim=3, verts=v, faces=[[0, 1, 2, 3], [0, 4, 1], [1, 4, 2], [2, 4, 3], [3, 4, 0]],
                  rounding=0.1, mass=1.0, inertia=[1.0, 1.0, 1.0])
    elif bad == "bowtie":
        sh = dict(W.square(1.0, 0.15), inertia=[1.0])
        sh["verts"] = np.array([[-.5, -.5], [.5, .5], [.5, -.5], [-.5, .5], [-.6, 0.0]])
    elif bad == "clockwise":
        sh = dict(W.l_shape2d(1.0, 0.15))
        sh["verts"] = sh["verts"][::-1].copy()
    elif bad == "fold":
        sh = dict(W.square(1.0, 0.15), inertia=[1.0])
        sh["verts"] = np.array([[-.5, -.5], [.5, -.5], [.5, .5], [.5, 0.0], [-.5, .5]])
    elif bad == "offcentre":
        sh["verts"] = sh["verts"] + 0.1
    elif bad == "rounding":
        sh["rounding"] = 0.0
    reason = {"inward": "enclosed volume", "flipped_face": "consistently oriented",
              "open": "not closed", "nonplanar": "not planar", "nonconvex_face": "not convex",
              "bowtie": "simple", "clockwise": "counter-clockwise", "fold": "folds back",
              "offcentre": "centred", "rounding": "rounding"}[bad]
    with pytest.raises(dem.DemError, match=reason):
        dem.dem_shape_info(sh)


@pytest.mark.parametrize("sizes", [[3, 0, 2], [0], []])
def test_create_rejects_empty_replicas(dem, sizes):
    """Empty inputs are refused during validation, before any device work."""
    box = np.full((max(len(sizes), 1), 3), 10.0)
    with pytest.raises(dem.DemError) as e:
        dem.dem_create([W.cube(1.0, 0.15)], 1.0, 0.0, box, np.asarray(sizes, np.int32),
                       dem.DEM_FP32_COMP)
    assert e.value.code == dem.DEM_ERR_ARG


def test_create_rejects_bad_box(dem):
    with pytest.raises(dem.DemError) as e:
        dem.dem_create([W.cube(1.0, 0.15)], 1.0, 0.0, np.array([[10.0, -1.0, 10.0]]),
                       np.array([4], np.int32), dem.DEM_FP32_COMP)
    assert e.value.code == dem.DEM_ERR_ARG
