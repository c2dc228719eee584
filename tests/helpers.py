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
}
