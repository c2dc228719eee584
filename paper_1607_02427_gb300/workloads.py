"""Seeded synthetic inputs for the rounded-polytope DEM: shapes, lattices,
orientations, velocities and contact-rich random clusters.

Both the CUDA library's callers (bench, GPU tests) and the FP64 oracle's
callers (CPU tests, CPU baseline) take their inputs from here, and from
nowhere else.  The module therefore holds none of the method's arithmetic:
no feature nearest points, no pair potential, no force, no integrator.  What
it does hold is input data and input recipes:

* shape tables in each shape's principal-axis body frame (vertices, convex
  faces listed counter-clockwise seen from outside, rounding radius, mass,
  principal moments of inertia of the uniform inner solid in closed form),
  convex or concave (the L-shaped hexagon, the dented cube);
* the outer (rounded) volume or area of each shape in closed form, which
  turns a packing fraction into a box size (Steiner's formula for the
  parallel body at distance equal to the rounding radius);
* simple-cubic and face-centred-cubic lattices, uniform random orientations
  (Shoemake's method), Maxwell velocities and angular momenta;
* a random sequential placement that puts particles next to one another at
  prescribed separating-axis gaps, so that force tests see many contacts.

Units are reduced: lengths in the shape's edge length, energies in epsilon,
mass m = 1.  Every generator takes a numpy ``Generator`` or a config index;
the base seed of the named workloads is ``BASE_SEED + config_index``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 1607_02427
WCA_CUT = 2.0 ** (1.0 / 6.0)   # r_cut / sigma of the WCA potential (input recipe only)


# ---------------------------------------------------------------------------
# Shape tables
# ---------------------------------------------------------------------------

def _shape(dim, verts, faces, rounding, inertia, inner_measure, boundary, wedge,
           name):
    verts = np.ascontiguousarray(np.asarray(verts, dtype=np.float64).reshape(-1, dim))
    return {
        "name": name,
        "dim": dim,
        "verts": verts,
        "faces": None if faces is None else [list(map(int, f)) for f in faces],
        "rounding": float(rounding),
        "mass": 1.0,
        "inertia": np.asarray(inertia, dtype=np.float64),
        # closed-form measures used only to size boxes from a packing fraction
        "inner_measure": float(inner_measure),   # area (2D) or volume (3D)
        "boundary": float(boundary),             # perimeter (2D) or surface (3D)
        "wedge": float(wedge),                   # 3D: sum_e l_e (pi - alpha_e) / 2
    }


def square(edge: float = 1.0, rounding: float = 0.15):
    """Rounded square (2D), vertices counter-clockwise; I_z = m a^2 / 6."""
    h = 0.5 * edge
    verts = [(-h, -h), (h, -h), (h, h), (-h, h)]
    return _shape(2, verts, None, rounding, [edge * edge / 6.0],
                  edge * edge, 4 * edge, 0.0, "square")


def disk(rounding: float = 0.5, inertia: float = 0.0):
    """One-vertex 2D shape: a disk of radius ``rounding`` (sphere limit)."""
    return _shape(2, [(0.0, 0.0)], None, rounding, [inertia], 0.0, 0.0, 0.0, "disk")


def rod2d(length: float = 1.0, rounding: float = 0.15):
    """Two-vertex 2D shape with one edge (a 2D spherocylinder)."""
    h = 0.5 * length
    return _shape(2, [(-h, 0.0), (h, 0.0)], None, rounding, [length * length / 12.0],
                  0.0, 2 * length, 0.0, "rod2d")


def polygon(n: int, circumradius: float = 1.0, rounding: float = 0.15):
    """Regular n-gon (2D), counter-clockwise, centred; uniform lamina inertia."""
    ang = 2 * np.pi * np.arange(n) / n
    verts = np.stack([circumradius * np.cos(ang), circumradius * np.sin(ang)], 1)
    side = 2 * circumradius * math.sin(math.pi / n)
    area = 0.5 * n * circumradius ** 2 * math.sin(2 * math.pi / n)
    # polar moment of a regular polygon lamina about its centre (m = 1)
    iz = (circumradius ** 2 / 6.0) * (1 + 2 * math.cos(math.pi / n) ** 2)
    return _shape(2, verts, None, rounding, [iz], area, n * side, 0.0, f"polygon{n}")


def sphere(rounding: float = 0.5, inertia: float = 0.0):
    """One-vertex 3D shape: a sphere of radius ``rounding`` (sphere limit)."""
    return _shape(3, [(0.0, 0.0, 0.0)], None, rounding, [inertia] * 3, 0.0, 0.0, 0.0,
                  "sphere")


def cube(edge: float = 1.0, rounding: float = 0.15):
    """Rounded cube; faces counter-clockwise seen from outside; I = m a^2/6."""
    h = 0.5 * edge
    verts = [(-h, -h, -h), (h, -h, -h), (h, h, -h), (-h, h, -h),
             (-h, -h, h), (h, -h, h), (h, h, h), (-h, h, h)]
    faces = [(0, 3, 2, 1),   # z = -h
             (4, 5, 6, 7),   # z = +h
             (0, 1, 5, 4),   # y = -h
             (2, 3, 7, 6),   # y = +h
             (0, 4, 7, 3),   # x = -h
             (1, 2, 6, 5)]   # x = +h
    a2 = edge * edge
    return _shape(3, verts, faces, rounding, [a2 / 6.0] * 3, edge ** 3, 6 * a2,
                  12 * edge * (math.pi / 2) / 2, "cube")


def tetrahedron(edge: float = 1.0, rounding: float = 0.15):
    """Regular tetrahedron centred on its centroid; I = m a^2 / 20."""
    s = edge / (2.0 * math.sqrt(2.0))
    verts = [(s, s, s), (s, -s, -s), (-s, s, -s), (-s, -s, s)]
    faces = [(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)]
    dihedral = math.acos(1.0 / 3.0)
    return _shape(3, verts, faces, rounding, [edge * edge / 20.0] * 3,
                  edge ** 3 / (6 * math.sqrt(2)), math.sqrt(3) * edge * edge,
                  6 * edge * (math.pi - dihedral) / 2, "tetrahedron")


def octahedron(circumradius: float = 1.0, rounding: float = 0.1):
    """Regular octahedron with vertices at +-R e_k; I = m R^2 / 5."""
    r = circumradius
    verts = [(r, 0, 0), (-r, 0, 0), (0, r, 0), (0, -r, 0), (0, 0, r), (0, 0, -r)]
    faces = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4),
             (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    edge = math.sqrt(2) * r
    dihedral = math.acos(-1.0 / 3.0)
    return _shape(3, verts, faces, rounding, [r * r / 5.0] * 3,
                  4.0 * r ** 3 / 3.0, 2 * math.sqrt(3) * edge * edge,
                  12 * edge * (math.pi - dihedral) / 2, "octahedron")


def triangular_prism(side: float = 1.0, length: float = 1.0, rounding: float = 0.15):
    """Right prism on an equilateral triangle, centroid at the origin, axis z.

    Principal moments (m = 1): I_z = a^2/12, I_x = I_y = a^2/24 + h^2/12.
    """
    a, h = side, length
    rc = a / math.sqrt(3.0)           # triangle circumradius
    tri = [(0.0, rc), (-0.5 * a, -0.5 * rc), (0.5 * a, -0.5 * rc)]
    verts = [(x, y, -0.5 * h) for x, y in tri] + [(x, y, 0.5 * h) for x, y in tri]
    faces = [(0, 2, 1), (3, 4, 5), (1, 2, 5, 4), (2, 0, 3, 5), (0, 1, 4, 3)]
    tri_area = math.sqrt(3) / 4 * a * a
    wedge = 6 * a * (math.pi / 2) / 2 + 3 * h * (math.pi - math.pi / 3) / 2
    return _shape(3, verts, faces, rounding,
                  [a * a / 24 + h * h / 12, a * a / 24 + h * h / 12, a * a / 12],
                  tri_area * h, 2 * tri_area + 3 * a * h, wedge, "prism")


def icosahedron(edge: float = 1.0, rounding: float = 0.15):
    """Regular icosahedron (12 V / 30 E / 20 F); I = m (phi^2/10) a^2 ... closed form."""
    p = (1 + math.sqrt(5)) / 2
    s = edge / 2.0
    raw = []
    for a in (-1, 1):
        for b in (-1, 1):
            raw += [(0, a, b * p), (a, b * p, 0), (b * p, 0, a)]
    verts = np.array(raw, dtype=np.float64) * s
    # faces: all vertex triples at mutual distance == edge, oriented outward
    n = len(verts)
    faces = []
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                if all(abs(np.linalg.norm(verts[u] - verts[v]) - edge) < 1e-9
                       for u, v in ((i, j), (j, k), (i, k))):
                    nrm = np.cross(verts[j] - verts[i], verts[k] - verts[i])
                    faces.append((i, j, k) if nrm @ verts[i] > 0 else (i, k, j))
    vol = 5 * (3 + math.sqrt(5)) / 12 * edge ** 3
    dihedral = math.acos(-math.sqrt(5) / 3)
    # solid icosahedron about its centre: I = m a^2 (phi^2) / 10
    i0 = edge * edge * p * p / 10.0
    return _shape(3, verts, faces, rounding, [i0] * 3, vol, 5 * math.sqrt(3) * edge ** 2,
                  30 * edge * (math.pi - dihedral) / 2, "icosahedron")


def icosphere(radius: float = 1.0, rounding: float = 0.1):
    """Geodesic sphere: the regular icosahedron with every edge split at its
    midpoint and the new vertices pushed out to the circumsphere (42 V / 120 E
    / 80 F, triangles).  More features than one 32-bit mask holds: shapes
    like it take the two-level masks.  The icosahedral symmetry makes every
    axis principal (isotropic inertia of the uniform inner solid)."""
    ico = icosahedron(1.0, rounding)
    v = [np.asarray(x) / np.linalg.norm(x) for x in ico["verts"]]
    mid = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            m = v[a] + v[b]
            v.append(m / np.linalg.norm(m))
            mid[key] = len(v) - 1
        return mid[key]

    faces = []
    for a, b, c in ico["faces"]:
        ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    verts = np.array(v) * radius
    vol, cen, inertia = polyhedron_mass_properties(verts, faces)
    verts = verts - cen
    area = sum(0.5 * np.linalg.norm(np.cross(verts[b] - verts[a], verts[c] - verts[a]))
               for a, b, c in faces)
    # sum over edges of l_e (pi - alpha_e) / 2, alpha_e the interior dihedral angle
    normal = [np.cross(verts[b] - verts[a], verts[c] - verts[a]) for a, b, c in faces]
    normal = [nn / np.linalg.norm(nn) for nn in normal]
    edge_faces = {}
    for k, f in enumerate(faces):
        for u, w in zip(f, f[1:] + f[:1]):
            edge_faces.setdefault((min(u, w), max(u, w)), []).append(k)
    wedge = 0.0
    for (u, w), (f1, f2) in edge_faces.items():
        bend = math.acos(max(-1.0, min(1.0, float(normal[f1] @ normal[f2]))))   # pi - alpha_e
        wedge += np.linalg.norm(verts[u] - verts[w]) * bend / 2.0
    sh = _shape(3, verts, faces, rounding, np.diag(inertia), vol, area, wedge, "icosphere")
    return sh


# ---- concave shapes (Section "Model": the inner shape may be concave) -------
#
# Mass properties of a general polygon or polyhedron (uniform density, m = 1)
# from the divergence theorem: shoelace sums over the edges in 2D, signed
# tetrahedra (origin, face fan triangle) in 3D.  These size and centre the
# input shapes only.

def polygon_mass_properties(verts):
    """Area, centroid and polar moment about the centroid (per unit mass) of
    a simple counter-clockwise polygon."""
    v = np.asarray(verts, np.float64)
    w = np.roll(v, -1, axis=0)
    cr = v[:, 0] * w[:, 1] - w[:, 0] * v[:, 1]
    area = cr.sum() / 2.0
    cen = ((v + w) * cr[:, None]).sum(0) / (6.0 * area)
    sx = v[:, 0] ** 2 + v[:, 0] * w[:, 0] + w[:, 0] ** 2
    sy = v[:, 1] ** 2 + v[:, 1] * w[:, 1] + w[:, 1] ** 2
    j0 = (cr * (sx + sy)).sum() / 12.0           # integral of x^2 + y^2 about the origin
    return float(area), cen, float(j0 / area - cen @ cen)


def polyhedron_mass_properties(verts, faces):
    """Volume, centroid and inertia tensor about the centroid (per unit mass)
    of a closed polyhedron with faces counter-clockwise seen from outside."""
    v = np.asarray(verts, np.float64)
    vol, first, second = 0.0, np.zeros(3), np.zeros((3, 3))
    for f in faces:
        for k in range(1, len(f) - 1):
            a, b, c = v[f[0]], v[f[k]], v[f[k + 1]]
            det = float(a @ np.cross(b, c))
            s = a + b + c
            vol += det / 6.0
            first += det / 24.0 * s
            second += det / 120.0 * (np.outer(a, a) + np.outer(b, b) + np.outer(c, c)
                                     + np.outer(s, s))
    cen = first / vol
    cov = second / vol - np.outer(cen, cen)      # integral of x x^T per unit mass
    return vol, cen, np.trace(cov) * np.eye(3) - cov


def l_shape2d(arm: float = 1.0, rounding: float = 0.15):
    """L-shaped hexagon (2D, one reflex vertex): the 2a x 2a square minus its
    upper-right a x a quarter, centred on its centroid (5a/6, 5a/6 from the
    outer corner); I_z = 11 m a^2 / 18.  Packing fractions of this shape count
    its rounded convex hull (the pentagon with the notch filled in)."""
    a = arm
    raw = np.array([(0, 0), (2 * a, 0), (2 * a, a), (a, a), (a, 2 * a), (0, 2 * a)], np.float64)
    area, cen, iz = polygon_mass_properties(raw)
    hull_area = 3.5 * a * a
    hull_perimeter = 6 * a + math.sqrt(2) * a
    sh = _shape(2, raw - cen, None, rounding, [iz], hull_area, hull_perimeter, 0.0, "lshape")
    sh["area"] = area
    sh["reflex_vertex"] = 3
    return sh


def dented_cube(edge: float = 1.0, depth: float = 0.5, rounding: float = 0.15):
    """Cube whose top face is pushed in to a square pyramid of the given
    depth (concave; 9 vertices, 16 edges, 9 convex faces: the bottom, four
    sides and four triangles meeting at the apex on the axis).  Centred on
    its centre of mass; principal axes x, y, z by the four-fold symmetry.
    Packing fractions of this shape count its rounded convex hull (the cube)."""
    h = 0.5 * edge
    raw = [(-h, -h, -h), (h, -h, -h), (h, h, -h), (-h, h, -h),
           (-h, -h, h), (h, -h, h), (h, h, h), (-h, h, h), (0.0, 0.0, h - depth)]
    faces = [(0, 3, 2, 1), (0, 1, 5, 4), (2, 3, 7, 6), (0, 4, 7, 3), (1, 2, 6, 5),
             (4, 5, 8), (5, 6, 8), (6, 7, 8), (7, 4, 8)]
    vol, cen, inertia = polyhedron_mass_properties(raw, faces)
    a2 = edge * edge
    sh = _shape(3, np.asarray(raw) - cen, faces, rounding, np.diag(inertia), edge ** 3, 6 * a2,
                12 * edge * (math.pi / 2) / 2, "dented_cube")
    sh["volume"] = vol
    sh["apex"] = 8
    return sh


def circumradius(shape) -> float:
    return float(np.max(np.linalg.norm(shape["verts"], axis=1)))


def outer_measure(shape) -> float:
    """Area (2D) or volume (3D) of the rounded shape (Steiner's formula)."""
    r = shape["rounding"]
    if shape["dim"] == 2:
        return shape["inner_measure"] + shape["boundary"] * r + math.pi * r * r
    return (shape["inner_measure"] + shape["boundary"] * r + shape["wedge"] * r * r
            + 4.0 / 3.0 * math.pi * r ** 3)


def wca_cut(shape_a, shape_b, sigma: float = 0.0) -> float:
    """WCA cutoff for a shape pair (sigma_ij = r_a + r_b unless ``sigma`` > 0)."""
    s = sigma if sigma > 0 else shape_a["rounding"] + shape_b["rounding"]
    return WCA_CUT * s


# ---------------------------------------------------------------------------
# Orientations and velocities
# ---------------------------------------------------------------------------

def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform unit quaternions (w, x, y, z), Shoemake's subgroup algorithm."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], 1)
    q[q[:, 0] < 0] *= -1.0
    return q


def _rotmat(q):
    """Rotation matrices of unit quaternions (w, x, y, z), shape (n, 3, 3)."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def maxwell_velocities(rng, n_per_replica: Sequence[int], dim: int, kT: float,
                       mass: np.ndarray) -> np.ndarray:
    """v ~ N(0, kT/m) per component, centre-of-mass momentum removed per replica."""
    out = []
    off = 0
    for n in n_per_replica:
        m = mass[off:off + n, None]
        v = rng.normal(size=(n, dim)) * np.sqrt(kT / m)
        p = (m * v).sum(0) / m.sum()
        out.append(v - p)
        off += n
    return np.concatenate(out, 0)


def thermal_angmom(rng, inertia: np.ndarray, orient: np.ndarray, dim: int,
                   kT: float) -> np.ndarray:
    """World-frame angular momenta: body components ~ N(0, I_k kT), rotated to world."""
    n = len(inertia)
    if dim == 2:
        return (rng.normal(size=n) * np.sqrt(kT * inertia[:, 0])).reshape(n, 1)
    lb = rng.normal(size=(n, 3)) * np.sqrt(kT * inertia)
    return np.einsum("nij,nj->ni", _rotmat(orient), lb)


# ---------------------------------------------------------------------------
# Systems
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class System:
    """A batch of independent periodic replica systems (one or many)."""
    dim: int
    shapes: List[dict]
    shape_id: np.ndarray          # (N,) int32
    pos: np.ndarray               # (N, dim) float64, in [0, L) of the replica's box
    orient: np.ndarray            # 3D: (N, 4) quaternion w,x,y,z; 2D: (N, 1) angle
    vel: np.ndarray               # (N, dim)
    angmom: np.ndarray            # 3D: (N, 3) world frame; 2D: (N, 1)
    box: np.ndarray               # (R, dim) box of each replica
    replica_sizes: np.ndarray     # (R,) int32
    epsilon: float = 1.0
    sigma: float = 0.0            # <= 0: sigma_ij = rounding_i + rounding_j
    target_box: Optional[np.ndarray] = None   # box after compression, if any
    name: str = ""
    params: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(len(self.shape_id))

    @property
    def n_replicas(self) -> int:
        return int(len(self.replica_sizes))

    def replica_slices(self):
        off = np.concatenate([[0], np.cumsum(self.replica_sizes)])
        return [slice(int(off[k]), int(off[k + 1])) for k in range(self.n_replicas)]

    def replica(self, k: int) -> "System":
        s = self.replica_slices()[k]
        used = np.unique(self.shape_id[s])
        remap = {int(u): i for i, u in enumerate(used)}
        return System(self.dim, [self.shapes[int(u)] for u in used],
                      np.array([remap[int(u)] for u in self.shape_id[s]], np.int32),
                      self.pos[s].copy(), self.orient[s].copy(), self.vel[s].copy(),
                      self.angmom[s].copy(), self.box[k:k + 1].copy(),
                      np.array([s.stop - s.start], np.int32), self.epsilon, self.sigma,
                      None if self.target_box is None else self.target_box[k:k + 1].copy(),
                      f"{self.name}[{k}]", dict(self.params))

    def inertia(self) -> np.ndarray:
        return np.stack([self.shapes[int(s)]["inertia"] for s in self.shape_id], 0)

    def masses(self) -> np.ndarray:
        return np.array([self.shapes[int(s)]["mass"] for s in self.shape_id])


def _finish(rng, dim, shapes, shape_id, pos, box, sizes, kT, orient=None, **kw):
    n = len(shape_id)
    if orient is None:
        orient = (random_quaternions(rng, n) if dim == 3
                  else rng.uniform(-np.pi, np.pi, size=(n, 1)))
    sysm = System(dim, shapes, np.asarray(shape_id, np.int32),
                  np.ascontiguousarray(pos, dtype=np.float64), orient,
                  np.zeros((n, dim)), np.zeros((n, 3 if dim == 3 else 1)),
                  np.asarray(box, np.float64).reshape(-1, dim),
                  np.asarray(sizes, np.int32), **kw)
    sysm.vel = maxwell_velocities(rng, sizes, dim, kT, sysm.masses())
    sysm.angmom = thermal_angmom(rng, sysm.inertia(), orient, dim, kT)
    return sysm


def sc_sites(counts: Sequence[int], spacing: Sequence[float]) -> np.ndarray:
    """Cell-centred simple-cubic (or square) lattice sites."""
    axes = [(np.arange(c) + 0.5) * s for c, s in zip(counts, spacing)]
    grid = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in grid], 1)


def fcc_sites(counts: Sequence[int], a: float) -> np.ndarray:
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 0.25
    cells = sc_sites(counts, [1.0, 1.0, 1.0]) - 0.5
    return ((cells[:, None, :] + basis[None]) * a).reshape(-1, 3)


def safe_spacing(shape, sigma: float = 0.0) -> float:
    """Lattice spacing at which bounding spheres are one WCA cutoff apart."""
    return 2 * circumradius(shape) + wca_cut(shape, shape, sigma)


# ---- the five named workloads ------------------------------------------------

def config_squares_2d(n_side: int = 16, kT: float = 1.0, seed_index: int = 0) -> System:
    """256 rounded squares (edge 1, rounding 0.15, sigma 0.3), area fraction 0.5,
    square lattice start, uniform random angles, Maxwell velocities, NVE."""
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + seed_index))
    sh = square(1.0, 0.15)
    n = n_side * n_side
    L = math.sqrt(n * outer_measure(sh) / 0.5)
    s = L / n_side
    assert s >= safe_spacing(sh), "square lattice start would overlap"
    pos = sc_sites([n_side, n_side], [s, s])
    return _finish(rng, 2, [sh], np.zeros(n, np.int32), pos, [[L, L]], [n], kT,
                   epsilon=1.0, sigma=0.3, name="squares2d_N256_phi0.50",
                   params=dict(dt=1e-3, steps=1000, ensemble="nve", kT=kT))


def _compressible_sc(rng, sh, counts, phi, n_use=None, sigma=0.0):
    """SC sites in a box sized for ``phi``; if the target spacing is below the
    bounding-sphere-safe spacing, the start uses the safe spacing (zero energy,
    any orientation) and ``target`` records the box to compress to."""
    counts = list(counts)
    n_sites = int(np.prod(counts))
    n = n_sites if n_use is None else n_use
    vol = n * outer_measure(sh) / phi
    aspect = np.array(counts, np.float64) / counts[0]
    L0 = (vol / np.prod(aspect)) ** (1.0 / 3.0) * aspect
    s_target = L0[0] / counts[0]
    s0 = max(s_target, safe_spacing(sh, sigma))
    start = np.array(counts, np.float64) * s0
    sites = sc_sites(counts, [s0] * 3)
    if n < n_sites:
        sites = sites[np.sort(rng.choice(n_sites, size=n, replace=False))]
    return sites, start, L0


def config_cubes_4096(kT: float = 1.0, seed_index: int = 1, n_side: int = 16) -> System:
    """4096 rounded cubes (edge 1, rounding 0.15, sigma 0.3), phi = 0.40, SC start."""
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + seed_index))
    sh = cube(1.0, 0.15)
    pos, start, target = _compressible_sc(rng, sh, [n_side] * 3, 0.40, sigma=0.3)
    n = len(pos)
    return _finish(rng, 3, [sh], np.zeros(n, np.int32), pos, [start], [n], kT,
                   epsilon=1.0, sigma=0.3, target_box=target.reshape(1, 3),
                   name=f"cubes_N{n}_phi0.40",
                   params=dict(dt=1e-3, steps=10000, ensemble="nvt", kT=kT, tau_T=0.5))


def config_octahedra(cells=(32, 32, 64), kT: float = 1.0, seed_index: int = 2) -> System:
    """Rounded octahedra (circumradius 1, rounding 0.1, sigma 0.2), phi = 0.50,
    FCC cells in a 1:1:2 orthorhombic box (262,144 at the default size)."""
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + seed_index))
    sh = octahedron(1.0, 0.1)
    n = 4 * int(np.prod(cells))
    a_target = (4 * outer_measure(sh) / 0.50) ** (1.0 / 3.0)
    nn_safe = safe_spacing(sh, 0.2)
    a0 = max(a_target, nn_safe * math.sqrt(2))
    pos = fcc_sites(cells, a0)
    start = np.array(cells, np.float64) * a0
    target = np.array(cells, np.float64) * a_target
    return _finish(rng, 3, [sh], np.zeros(n, np.int32), pos, [start], [n], kT,
                   epsilon=1.0, sigma=0.2, target_box=target.reshape(1, 3),
                   name=f"octahedra_N{n}_phi0.50",
                   params=dict(dt=5e-4, steps=100000, ensemble="nve", kT=kT))


def config_batched(n_replicas: int = 512, n_lo: int = 128, n_hi: int = 2048,
                   kT: float = 1.0, seed_index: int = 3) -> System:
    """Independent replicas: N_k ~ U{n_lo..n_hi}, shape k mod 3 = cube /
    tetrahedron / triangular prism (edge 1), rounding r_k ~ U[0.1, 0.2],
    sigma_k = 2 r_k, packing fraction phi_k ~ U[0.30, 0.55], cubic boxes, a
    seeded random subset of ceil(N^(1/3))^3 simple-cubic sites."""
    ss = np.random.SeedSequence(BASE_SEED + seed_index)
    top = np.random.default_rng(ss)
    kids = ss.spawn(n_replicas)
    sizes = top.integers(n_lo, n_hi + 1, size=n_replicas)
    rounding = top.uniform(0.1, 0.2, size=n_replicas)
    phis = top.uniform(0.30, 0.55, size=n_replicas)
    makers = [cube, tetrahedron, triangular_prism]
    shapes, pos, starts, targets, ids, ors, vel, am = [], [], [], [], [], [], [], []
    for k in range(n_replicas):
        rng = np.random.default_rng(kids[k])
        sh = makers[k % 3](1.0, rounding=float(rounding[k])) if k % 3 != 2 else \
            triangular_prism(1.0, 1.0, rounding=float(rounding[k]))
        n = int(sizes[k])
        m = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
        sites, start, target = _compressible_sc(rng, sh, [m] * 3, float(phis[k]), n_use=n)
        sub = _finish(rng, 3, [sh], np.zeros(n, np.int32), sites, [start], [n], kT)
        shapes.append(sh)
        ids.append(np.full(n, k, np.int32))
        pos.append(sub.pos), ors.append(sub.orient), vel.append(sub.vel), am.append(sub.angmom)
        starts.append(start), targets.append(target)
    return System(3, shapes, np.concatenate(ids), np.concatenate(pos), np.concatenate(ors),
                  np.concatenate(vel), np.concatenate(am), np.array(starts),
                  sizes.astype(np.int32), 1.0, 0.0, np.array(targets),
                  name=f"batched_R{n_replicas}_N{n_lo}-{n_hi}",
                  params=dict(dt=1e-3, ensemble="nvt", kT=kT, tau_T=0.5,
                              phi=phis.tolist()))


def config_large(counts=(64, 128, 128), kT: float = 1.0, seed_index: int = 4) -> System:
    """Rounded cubes (edge 1, rounding 0.15, sigma 0.3), phi = 0.55, SC start in a
    1:2:2 orthorhombic box (1,048,576 at the default size)."""
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + seed_index))
    sh = cube(1.0, 0.15)
    pos, start, target = _compressible_sc(rng, sh, counts, 0.55, sigma=0.3)
    n = len(pos)
    return _finish(rng, 3, [sh], np.zeros(n, np.int32), pos, [start], [n], kT,
                   epsilon=1.0, sigma=0.3, target_box=target.reshape(1, 3),
                   name=f"cubes_N{n}_phi0.55",
                   params=dict(dt=1e-3, steps=1000, ensemble="nvt", kT=kT, tau_T=0.5))


PAPER_TABLE_SHAPES = ("sphere", "cube", "icosahedron")


def config_paper_table(shape: str = "icosahedron", n: int = 65536, phi: float = 0.45,
                       kT: float = 1.0, seed_index: int = 5) -> System:
    """One dense-fluid system of the paper's performance table (Section
    "Performance": spheres with the central WCA, cubes and icosahedra, N = 256,
    4096 or 65,536).  The paper gives no density, size or rounding for these
    runs; here: packing fraction 0.45 of the rounded volume, sphere diameter
    sigma = 1 (rounding 0.5), cube and icosahedron edge 1 with rounding 0.15
    (sigma = 0.3), a seeded subset of ceil(N^(1/3))^3 simple-cubic sites,
    compressed from the safe spacing like the other 3D configs; NVT kT = 1."""
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + seed_index))
    makers = {"sphere": lambda: sphere(0.5), "cube": lambda: cube(1.0, 0.15),
              "icosahedron": lambda: icosahedron(1.0, 0.15)}
    sh = makers[shape]()
    m = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    pos, start, target = _compressible_sc(rng, sh, [m] * 3, phi, n_use=n)
    return _finish(rng, 3, [sh], np.zeros(n, np.int32), pos, [start], [n], kT,
                   epsilon=1.0, sigma=0.0, target_box=target.reshape(1, 3),
                   name=f"{shape}s_N{n}_phi{phi:.2f}",
                   params=dict(dt=1e-3, ensemble="nvt", kT=kT, tau_T=0.5))


def config_energy_drift(shape: str = "tetrahedron", n_side: int = 8, phi: float = 0.4,
                        kT: float = 1.0, seed_index: int = 6) -> System:
    """The fluids of Section "Energy Conservation", in reduced units with
    sigma = 1 (rounding 0.5): squares of edge 4.24 sigma (2D, n_side^2
    particles on a square lattice) or tetrahedra of edge 8.49 sigma (3D,
    n_side^3 particles compressed from the safe lattice spacing), at packing
    fraction ``phi`` of the rounded shapes (the paper gives no density;
    0.5 for squares and 0.4 for tetrahedra are this reading's fluids)."""
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + seed_index))
    if shape == "square":
        sh = square(4.24, 0.5)
        n = n_side * n_side
        L = math.sqrt(n * outer_measure(sh) / phi)
        s = L / n_side
        assert s >= safe_spacing(sh), "square lattice start would overlap"
        pos = sc_sites([n_side, n_side], [s, s])
        return _finish(rng, 2, [sh], np.zeros(n, np.int32), pos, [[L, L]], [n], kT,
                       epsilon=1.0, sigma=0.0, name=f"drift_squares_N{n}_phi{phi:.2f}",
                       params=dict(dt=0.01, ensemble="nve", kT=kT))
    sh = tetrahedron(8.49, 0.5)
    pos, start, target = _compressible_sc(rng, sh, [n_side] * 3, phi)
    n = len(pos)
    return _finish(rng, 3, [sh], np.zeros(n, np.int32), pos, [start], [n], kT,
                   epsilon=1.0, sigma=0.0, target_box=target.reshape(1, 3),
                   name=f"drift_tetrahedra_N{n}_phi{phi:.2f}",
                   params=dict(dt=0.01, ensemble="nve", kT=kT))


def sample_like(system: System, n_target: int = 512, kT: float = 1.0, seed: int = 0) -> System:
    """A small system like replica 0 of ``system``: the same shapes (drawn in
    the replica's proportions) at its target density, on m^d simple-cubic
    sites in a cubic box (m = round(n_target^(1/d))); for timing the CPU oracle
    on workloads too large for it."""
    rep = system.replica(0)
    dim = rep.dim
    box = rep.target_box[0] if rep.target_box is not None else rep.box[0]
    rho = rep.n / float(np.prod(np.asarray(box, np.float64)[:dim]))
    m = max(2, int(round(n_target ** (1.0 / dim))))
    n = m ** dim
    L = (n / rho) ** (1.0 / dim)
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + 900 + seed))
    ids = rep.shape_id[rng.integers(0, rep.n, size=n)]
    pos = sc_sites([m] * dim, [L / m] * dim)
    return _finish(rng, dim, rep.shapes, ids, pos, [[L] * dim], [n], kT,
                   epsilon=rep.epsilon, sigma=rep.sigma,
                   name=f"{rep.name}_sample{n}")


# ---------------------------------------------------------------------------
# Contact-rich random clusters (force tests)
# ---------------------------------------------------------------------------

def _support(shape, orient_row, direction):
    """max over vertices of (R v) . direction (the inner shape's support value)."""
    v = shape["verts"]
    if shape["dim"] == 2:
        c, s = math.cos(orient_row[0]), math.sin(orient_row[0])
        w = np.stack([c * v[:, 0] - s * v[:, 1], s * v[:, 0] + c * v[:, 1]], 1)
    else:
        w = v @ _rotmat(orient_row[None])[0].T
    return float(np.max(w @ direction))


def contact_cluster(shapes: List[dict], shape_id: Sequence[int], box: Sequence[float],
                    rng: np.random.Generator, gap=(0.85, 1.15), gap_min: float = 0.8,
                    sigma: float = 0.0, kT: float = 1.0, max_tries: int = 2000,
                    free: float = 0.1, name: str = "cluster") -> System:
    """Random sequential placement of particles next to earlier ones.

    Each new particle takes a uniform random orientation and sits along a
    random direction from a random earlier particle, at a separating-axis gap
    g ~ U[gap] * sigma_ij along that direction.  It is kept only if, along the
    centre line to every other particle (minimum image), the separating-axis
    gap is at least ``gap_min * sigma_ij``.  The separating-axis gap is a lower
    bound on the true inner-shape distance, so no feature pair starts closer
    than ``gap_min * sigma_ij``; many start within the WCA range.
    """
    dim = shapes[0]["dim"]
    box = np.asarray(box, np.float64)
    shape_id = np.asarray(shape_id, np.int32)
    n = len(shape_id)
    orient = (random_quaternions(rng, n) if dim == 3
              else rng.uniform(-np.pi, np.pi, size=(n, 1)))
    pos = np.zeros((n, dim))
    radii = np.array([circumradius(shapes[s]) for s in shape_id])
    rnd = np.array([shapes[s]["rounding"] for s in shape_id])
    pos[0] = rng.random(dim) * box
    placed = 1
    for i in range(1, n):
        for _ in range(max_tries):
            if free > 0 and rng.random() < free:
                x = rng.random(dim) * box      # a free placement starts a new cluster
            else:
                a = int(rng.integers(placed))
                u = rng.normal(size=dim)
                u /= np.linalg.norm(u)
                sig = sigma if sigma > 0 else rnd[a] + rnd[i]
                t = (_support(shapes[shape_id[a]], orient[a], u)
                     + _support(shapes[shape_id[i]], orient[i], -u)
                     + rng.uniform(*gap) * sig)
                x = np.mod(pos[a] + t * u, box)
            ok = True
            d = pos[:placed] - x
            d -= box * np.round(d / box)
            dist = np.linalg.norm(d, axis=1)
            for k in np.nonzero(dist < radii[:placed] + radii[i] + 2.0 * WCA_CUT * 0.5 *
                                (rnd[:placed] + rnd[i]) + 1e-12)[0]:
                if dist[k] == 0.0:
                    ok = False
                    break
                e = d[k] / dist[k]
                sig_k = sigma if sigma > 0 else rnd[k] + rnd[i]
                g = dist[k] - _support(shapes[shape_id[k]], orient[k], -e) \
                    - _support(shapes[shape_id[i]], orient[i], e)
                if g < gap_min * sig_k:
                    ok = False
                    break
            if ok:
                pos[i] = x
                break
        else:
            raise RuntimeError("contact_cluster: could not place particle; lower density")
        placed += 1
    sysm = _finish(rng, dim, shapes, shape_id, pos, [box], [n], kT, orient=orient,
                   epsilon=1.0, sigma=sigma, name=name)
    return sysm


def merge(systems: Sequence[System], name: str = "merged") -> System:
    """Concatenate single- or multi-replica systems into one batch."""
    shapes, ids = [], []
    for s in systems:
        ids.append(s.shape_id + len(shapes))
        shapes += s.shapes
    cat = lambda f: np.concatenate([getattr(s, f) for s in systems], 0)
    tb = None
    if all(s.target_box is not None for s in systems):
        tb = cat("target_box")
    return System(systems[0].dim, shapes, np.concatenate(ids), cat("pos"), cat("orient"),
                  cat("vel"), cat("angmom"), cat("box"), cat("replica_sizes"),
                  systems[0].epsilon, systems[0].sigma, tb, name)


# ---------------------------------------------------------------------------
# Contact-rich lattice starts (full-size force tests)
# ---------------------------------------------------------------------------

def _axis_extents(shape, q):
    """Half extents of the rotated inner shape along x, y, z (support values
    along +-e_k, the larger of the two), for quaternions q (n, 4)."""
    w = np.einsum("nij,vj->nvi", _rotmat(q), shape["verts"])
    return np.abs(w).max(1)


def slab_lattice_start(system: System, gap: float = 0.85, tries: int = 24,
                       seed: int = 0) -> System:
    """Re-orient a simple-cubic lattice system so that neighbours are close
    but never closer than ``gap * sigma`` (3D).

    Sites of a simple-cubic lattice of spacing s differ by at least s along
    some axis, so the inner shapes of i and j are at least
    s - h_i - h_j apart along that axis, where h is the half extent of a
    rotated shape along the axis.  Each particle draws uniform random
    orientations until all three half extents are <= (s - gap sigma)/2; if
    none of ``tries`` draws passes it keeps the body-frame orientation, and
    if even that fails the replica's lattice is stretched until it passes.
    Positions are the replica's sites (the box is scaled with the lattice).
    """
    assert system.dim == 3
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + 97 + seed))
    # start from the lattice scaled to the target (compressed) box, if any
    box0 = system.box if system.target_box is None else system.target_box
    pos0 = system.pos.copy()
    if system.target_box is not None:
        for r, sl in enumerate(system.replica_slices()):
            pos0[sl] = system.pos[sl] * (system.target_box[r] / system.box[r])
    out = dataclasses.replace(system, pos=pos0, orient=system.orient.copy(),
                              box=np.array(box0, np.float64), target_box=None)
    system = dataclasses.replace(system, pos=pos0, box=np.array(box0, np.float64))
    for r, sl in enumerate(system.replica_slices()):
        sh = system.shapes[int(system.shape_id[sl.start])]
        sig = system.sigma if system.sigma > 0 else 2 * sh["rounding"]
        n = sl.stop - sl.start
        box = system.box[r]
        m = np.round(box / (box.min() / np.ceil(n ** (1 / 3) - 1e-9))).astype(int)
        m = np.maximum(m, 1)
        s = float(box[0] / m[0])
        ident = _axis_extents(sh, np.array([[1.0, 0, 0, 0]]))[0].max()
        need = 2 * ident + gap * sig
        if s < need:
            scale = need / s
            out.box[r] = box * scale
            out.pos[sl] = system.pos[sl] * scale
            s = need
        lim = 0.5 * (s - gap * sig)
        q = np.tile([1.0, 0, 0, 0], (n, 1))
        todo = np.arange(n)
        for _ in range(tries):
            if len(todo) == 0:
                break
            cand = random_quaternions(rng, len(todo))
            ok = _axis_extents(sh, cand).max(1) <= lim
            q[todo[ok]] = cand[ok]
            todo = todo[~ok]
        out.orient[sl] = q
    # angular momenta follow the new orientations (same body-frame draws)
    return out
