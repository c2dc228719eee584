"""Small shared test utilities (system construction, rotations for tests)."""
from __future__ import annotations

import numpy as np

from paper_1607_02427_gb300 import workloads as W


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def axis_angle_quat(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[np.cos(angle / 2)], np.sin(angle / 2) * axis])


def rotmat(q):
    return W._rotmat(np.asarray(q, float)[None])[0]


def two_body(shape_a, shape_b, d, qa=None, qb=None, box=50.0, sigma=0.0):
    """Two particles: a at the box centre, b at a + d."""
    dim = shape_a["dim"]
    c = np.full(dim, box / 2)
    pos = np.stack([c, c + np.asarray(d, float)])
    if dim == 3:
        orient = np.stack([qa if qa is not None else [1, 0, 0, 0],
                           qb if qb is not None else [1, 0, 0, 0]]).astype(float)
    else:
        orient = np.array([[qa or 0.0], [qb or 0.0]], float)
    shapes = [shape_a, shape_b]
    return W.System(dim, shapes, np.array([0, 1], np.int32), pos, orient,
                    np.zeros((2, dim)), np.zeros((2, 3 if dim == 3 else 1)),
                    np.full((1, dim), box), np.array([2], np.int32), 1.0, sigma)


def open_cluster(shapes, shape_id, seed, gap=(0.85, 1.15), gap_min=0.8, box=400.0, kT=1.0,
                 sigma=0.0):
    """A contact-rich cluster, unwrapped and centred in a large periodic box so
    that no pair interacts across the boundary."""
    rng = np.random.default_rng(seed)
    dim = shapes[0]["dim"]
    s = W.contact_cluster(shapes, shape_id, [box] * dim, rng, gap=gap, gap_min=gap_min,
                          sigma=sigma, kT=kT, free=0.0)
    d = s.pos - s.pos[0]
    d -= box * np.round(d / box)
    s.pos = d - d.mean(0) + box / 2
    return s


def copy_system(s, **over):
    import copy
    t = copy.copy(s)
    for k in ("pos", "orient", "vel", "angmom", "box"):
        setattr(t, k, np.array(getattr(s, k), copy=True))
    for k, v in over.items():
        setattr(t, k, v)
    return t


SHAPES_3D = {
    "cube": lambda: W.cube(1.0, 0.15),
    "tetrahedron": lambda: W.tetrahedron(1.0, 0.15),
    "octahedron": lambda: W.octahedron(1.0, 0.1),
    "prism": lambda: W.triangular_prism(1.0, 1.0, 0.15),
    "icosahedron": lambda: W.icosahedron(0.8, 0.15),
    # 42 V / 120 E / 80 F: beyond one 32-bit feature mask
    "icosphere": lambda: W.icosphere(0.7, 0.12),
}


def nest_guests(s, hosts, guest, local_points, seed, gap_min=0.8):
    """Append one-vertex guests (disks or spheres) at ``local_points`` (body
    frame of each host: e.g. inside an L-shape's notch or a dented cube's
    dent, within r_cut of the concave features).  A guest is kept only when,
    along the centre line to every particle but its host, the separating-axis
    gap is at least gap_min * sigma_ij.  Returns a new one-replica system."""
    rng = np.random.default_rng(seed)
    dim = s.dim
    box = s.box[0]
    shapes = list(s.shapes) + [guest]
    gid = len(shapes) - 1
    pos, orient = [s.pos.copy()], [s.orient.copy()]
    ids = [s.shape_id.copy()]
    added = []
    for h in hosts:
        lp = np.asarray(local_points[int(rng.integers(len(local_points)))], float)
        if dim == 3:
            x = s.pos[h] + rotmat(s.orient[h]) @ lp
        else:
            c, sn = np.cos(s.orient[h, 0]), np.sin(s.orient[h, 0])
            x = s.pos[h] + np.array([c * lp[0] - sn * lp[1], sn * lp[0] + c * lp[1]])
        x = np.mod(x, box)
        cand = np.concatenate([s.pos] + [np.array(added).reshape(-1, dim)], 0)
        cand_ids = np.concatenate([s.shape_id, np.full(len(added), gid, np.int32)])
        ok = True
        for k in range(len(cand)):
            if k == h:
                continue
            d = x - cand[k]
            d -= box * np.round(d / box)
            dist = np.linalg.norm(d)
            if dist == 0.0:
                ok = False
                break
            e = d / dist
            sh_k = shapes[int(cand_ids[k])]
            sig = sh_k["rounding"] + guest["rounding"] if s.sigma <= 0 else s.sigma
            if k < s.n:
                g = dist - W._support(sh_k, s.orient[k], e)
            else:
                g = dist                     # an earlier guest: a point

            if g < gap_min * sig:
                ok = False
                break
        if ok:
            added.append(x)
    m = len(added)
    if m == 0:
        raise RuntimeError("no guest could be placed")
    rng2 = np.random.default_rng(seed + 1)
    g_or = (np.tile([1.0, 0, 0, 0], (m, 1)) if dim == 3 else np.zeros((m, 1)))
    n = s.n + m
    out = W.System(dim, shapes, np.concatenate(ids + [np.full(m, gid, np.int32)]),
                   np.concatenate(pos + [np.array(added)], 0), np.concatenate(orient + [g_or], 0),
                   np.zeros((n, dim)), np.zeros((n, 3 if dim == 3 else 1)), s.box.copy(),
                   np.array([n], np.int32), s.epsilon, s.sigma, name=s.name + "+nested")
    out.vel = W.maxwell_velocities(rng2, [n], dim, 1.0, out.masses())
    out.angmom = W.thermal_angmom(rng2, out.inertia(), out.orient, dim, 1.0)
    return out


def notch_points(L, sigma, fracs=((0.85, 0.95), (0.9, 0.8), (0.97, 0.88))):
    """Body-frame points in an L-shape's notch at fractions of r_cut from the
    two edges that meet at the reflex vertex."""
    rc = 2.0 ** (1.0 / 6.0) * sigma
    c = L["verts"][L["reflex_vertex"]]
    return [c + rc * np.array(f) for f in fracs]


def dent_points(D, sigma, fracs=(0.82, 0.9, 0.97)):
    """Body-frame points on a dented cube's axis above the apex, the four dent
    faces at fractions of r_cut."""
    rc = 2.0 ** (1.0 / 6.0) * sigma
    apex = D["verts"][D["apex"]]
    t = 0.5 * (D["verts"][:, 0].max() - D["verts"][:, 0].min())
    depth = D["verts"][4, 2] - apex[2]
    k = np.hypot(depth, t) / t           # axial height per unit face distance
    return [apex + np.array([0.0, 0.0, f * rc * k]) for f in fracs]


# ---------------------------------------------------------------------------
# Aligned and tied geometries (Section "Model": the parallel-edge rule and the
# face-to-face overcounting example)
# ---------------------------------------------------------------------------

SIG_EDGE = 0.3            # sigma of the edge-case systems (rounding 0.15)


def ridge_pair(sin2, dx, gap, sigma=SIG_EDGE):
    """Two unit cubes, each turned 45 degrees about x so that an edge along x
    forms a ridge; i's ridge points up, j's down, at a height gap above it.
    j is turned further by theta about z (sin^2 theta = sin2: the squared
    sine of the angle between the two ridges) and shifted by dx along x.
    dx = 0.3: the ridges' projections overlap on [-0.2, 0.5], so the
    parallel-edge rule puts the contact at the overlap's midpoint x = 0.15,
    while the ordinary nearest points lie where the ridges cross, x = 0.3;
    dx = 1.2: no overlap (the rule falls back to the endpoint pairs)."""
    r45 = axis_angle_quat([1, 0, 0], np.pi / 4)
    th = np.arcsin(np.sqrt(sin2))
    qj = quat_mul(axis_angle_quat([0, 0, 1], th), r45)
    return two_body(W.cube(1.0, sigma / 2), W.cube(1.0, sigma / 2),
                    [dx, 0.0, np.sqrt(2.0) + gap], qa=r45, qb=qj, sigma=sigma)


def face_to_face(gap, lateral=(0.0, 0.0), sigma=SIG_EDGE):
    """Two aligned unit cubes, j above i's top face at the face gap, shifted
    sideways by lateral (partial face overlap when non-zero)."""
    return two_body(W.cube(1.0, sigma / 2), W.cube(1.0, sigma / 2),
                    [lateral[0], lateral[1], 1.0 + gap], sigma=sigma)


def collinear_ridges(gap, sigma=SIG_EDGE):
    """Two cubes turned 45 degrees about x, side by side along x: their
    ridges are collinear with a gap (parallel, no overlap) and their x faces
    face each other at the same gap."""
    r45 = axis_angle_quat([1, 0, 0], np.pi / 4)
    return two_body(W.cube(1.0, sigma / 2), W.cube(1.0, sigma / 2), [1.0 + gap, 0.0, 0.0],
                    qa=r45, qb=r45, sigma=sigma)


def vertex_over_face_edge(gap, corner=False, sigma=SIG_EDGE):
    """A cube j standing on a vertex whose lowest vertex lies a gap above
    i's top face, exactly over the edge y = 0.5 of that face (corner: over
    the corner x = y = 0.5): the vertex projects onto the face's boundary,
    where the inside test of the vertex-face term is tied."""
    a = np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)
    axis = np.cross(a, [0.0, 0.0, -1.0])
    ang = np.arccos(np.dot(a, [0.0, 0.0, -1.0]))
    qj = axis_angle_quat(axis, ang)
    low = rotmat(qj) @ np.array([0.5, 0.5, 0.5])          # the vertex that points down
    target = np.array([0.5 if corner else 0.0, 0.5, 0.5 + gap])
    return two_body(W.cube(1.0, sigma / 2), W.cube(1.0, sigma / 2), target - low, qb=qj,
                    sigma=sigma)


def aligned_lattice(dim, n_side, gap, jitter, seed, sigma=SIG_EDGE):
    """Unrotated unit squares or cubes on a square or simple-cubic lattice of
    spacing 1 + gap in a periodic box, each displaced by up to jitter per
    axis: every edge pair is exactly parallel or exactly perpendicular, and
    neighbours meet face to face (edge to edge in 2D) at gaps near gap with
    partial overlaps."""
    rng = np.random.default_rng(seed)
    a = 1.0 + gap
    sites = W.sc_sites([n_side] * dim, [a] * dim)
    pos = sites + rng.uniform(-jitter, jitter, size=sites.shape)
    n = len(pos)
    shape = W.cube(1.0, sigma / 2) if dim == 3 else W.square(1.0, sigma / 2)
    orient = np.tile([1.0, 0, 0, 0], (n, 1)) if dim == 3 else np.zeros((n, 1))
    s = W.System(dim, [shape], np.zeros(n, np.int32), np.mod(pos, n_side * a), orient,
                 np.zeros((n, dim)), np.zeros((n, 3 if dim == 3 else 1)),
                 np.full((1, dim), n_side * a), np.array([n], np.int32), 1.0, sigma)
    return s


def square_pairs_2d(gap, sigma=SIG_EDGE):
    """2D ties: squares corner to corner (each corner vertex at the two
    edges of the other corner) and edge to edge (facing edges parallel),
    as two replicas."""
    sq = W.square(1.0, sigma / 2)
    cc = two_body(sq, sq, [1 + gap / np.sqrt(2), 1 + gap / np.sqrt(2)], sigma=sigma)
    ee = two_body(sq, sq, [0.3, 1 + gap], sigma=sigma)
    return W.merge([cc, ee], "square_pairs")


def swap_pair(s):
    """The same two-particle system with the particles' order swapped (the
    parallel-edge rule's reference edge is the lower-indexed particle's)."""
    t = copy_system(s)
    for k in ("pos", "orient", "vel", "angmom"):
        setattr(t, k, getattr(t, k)[::-1].copy())
    t.shape_id = t.shape_id[::-1].copy()
    return t
