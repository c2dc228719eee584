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


@pytest.mark.parametrize("bad", ["inward", "nonconvex", "offcentre", "rounding"])
def test_shape_validation(dem, bad):
    sh = W.cube(1.0, 0.15)
    sh = dict(sh, inertia=None)
    if bad == "inward":
        sh["faces"] = [list(reversed(f)) for f in sh["faces"]]
    elif bad == "nonconvex":
        sh = dict(W.square(1.0, 0.15), inertia=None)
        sh["verts"] = np.array([[-.5, -.5], [.5, -.5], [0, -.3], [-.5, .5]])
    elif bad == "offcentre":
        sh["verts"] = sh["verts"] + 0.1
    elif bad == "rounding":
        sh["rounding"] = 0.0
    with pytest.raises(dem.DemError):
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
