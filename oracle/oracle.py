"""ctypes wrapper of the FP64 oracle (test infrastructure only).

Functions take a ``workloads.System``-like object (``dim``, ``shapes``,
``shape_id``, ``pos``, ``orient``, ``box`` ...) or plain arrays, and return
numpy arrays.  Multi-replica systems are evaluated one replica at a time:
replicas are independent periodic systems.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Squared-sine threshold of the parallel-edge rule (a reading: the paper says
# only "sufficiently close to parallel").
DEFAULT_PAR_EPS = 1e-6


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile dem_oracle.c with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o",
                               tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        dp, ip, lp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_longlong)
        lib.oracle_forces.restype = C.c_int
        lib.oracle_forces.argtypes = [C.c_int, C.c_int, ip, dp, ip, ip, ip, dp, C.c_double,
                                      C.c_double, C.c_double, C.c_int, ip, dp, dp, dp, dp, dp,
                                      dp, dp, dp, dp, ip, lp]
        lib.oracle_run.restype = C.c_int
        lib.oracle_run.argtypes = [C.c_int, C.c_int, ip, dp, ip, ip, ip, dp, dp, dp, C.c_double,
                                   C.c_double, C.c_double, C.c_int, ip, dp, dp, dp, dp, dp, dp,
                                   C.c_int, C.c_double, C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double, dp]
        lib.oracle_point_segment.restype = C.c_double
        lib.oracle_point_segment.argtypes = [dp, dp, dp, dp]
        lib.oracle_point_face.restype = C.c_double
        lib.oracle_point_face.argtypes = [dp, C.c_int, dp, dp]
        lib.oracle_segment_segment.restype = C.c_double
        lib.oracle_segment_segment.argtypes = [dp, dp, dp, dp, C.c_double, dp, dp, ip]
        lib.oracle_set_parallel.restype = None
        lib.oracle_set_parallel.argtypes = [C.c_int, C.c_int]
        lib.oracle_max_threads.restype = C.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_wca.restype = C.c_double
        lib.oracle_wca.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def pack_shapes(shapes):
    """Flatten shape dicts into the oracle's packed arrays."""
    vert_off, verts, sfo, fvo, fidx, rnd = [0], [], [0], [0], [], []
    for sh in shapes:
        v = np.asarray(sh["verts"], np.float64)
        if v.shape[1] == 2:
            v = np.concatenate([v, np.zeros((len(v), 1))], 1)
        verts.append(v)
        vert_off.append(vert_off[-1] + len(v))
        faces = sh.get("faces") or []
        for f in faces:
            fidx.extend(int(k) for k in f)
            fvo.append(len(fidx))
        sfo.append(sfo[-1] + len(faces))
        rnd.append(float(sh["rounding"]))
    return dict(vert_off=np.array(vert_off, np.int32),
                verts=np.concatenate(verts, 0).ravel(),
                shape_face_off=np.array(sfo, np.int32),
                face_vert_off=np.array(fvo, np.int32),
                face_idx=np.array(fidx if fidx else [0], np.int32),
                rounding=np.array(rnd, np.float64))


def forces(system, par_eps: float = DEFAULT_PAR_EPS, scales: bool = True):
    """Force, torque, per-particle energy, virial and term scales.

    Returns a dict with ``force`` (N, dim), ``torque`` (N, 3) in 3D or (N, 1)
    in 2D (world frame), ``energy`` (N,), ``virial`` (R, 3, 3) per replica,
    ``U`` (R,) per replica, ``fscale``/``tscale`` (N,), ``flags`` (N,) and
    ``counts`` (R, 3).
    """
    lib = _load()
    dim = system.dim
    n = system.n
    out = dict(force=np.zeros((n, dim)), torque=np.zeros((n, 3 if dim == 3 else 1)),
               energy=np.zeros(n), fscale=np.zeros(n), tscale=np.zeros(n),
               flags=np.zeros(n, np.int32), virial=np.zeros((system.n_replicas, 3, 3)),
               U=np.zeros(system.n_replicas), counts=np.zeros((system.n_replicas, 3), np.int64))
    pk = pack_shapes(system.shapes)
    keep = [pk]
    args_shape = []
    for k in ("vert_off",):
        a, p = _i(pk[k]); keep.append(a); args_shape.append(p)
    a, p = _d(pk["verts"]); keep.append(a); args_shape.append(p)
    for k in ("shape_face_off", "face_vert_off", "face_idx"):
        a, p = _i(pk[k]); keep.append(a); args_shape.append(p)
    a, p = _d(pk["rounding"]); keep.append(a); args_shape.append(p)
    orient = np.asarray(system.orient, np.float64)
    for r, sl in enumerate(system.replica_slices()):
        m = sl.stop - sl.start
        sid, sid_p = _i(system.shape_id[sl])
        pos, pos_p = _d(system.pos[sl])
        ori, ori_p = _d(orient[sl])
        box, box_p = _d(system.box[r])
        f = np.zeros((m, dim)); t = np.zeros((m, 3 if dim == 3 else 1)); e = np.zeros(m)
        vir = np.zeros(9); fs = np.zeros(m); ts = np.zeros(m)
        fl = np.zeros(m, np.int32); cnt = np.zeros(3, np.int64)
        rc = lib.oracle_forces(
            dim, len(system.shapes), *args_shape, float(system.epsilon), float(system.sigma),
            float(par_eps), m, sid_p, pos_p, ori_p, box_p,
            f.ctypes.data_as(C.POINTER(C.c_double)), t.ctypes.data_as(C.POINTER(C.c_double)),
            e.ctypes.data_as(C.POINTER(C.c_double)), vir.ctypes.data_as(C.POINTER(C.c_double)),
            fs.ctypes.data_as(C.POINTER(C.c_double)) if scales else None,
            ts.ctypes.data_as(C.POINTER(C.c_double)) if scales else None,
            fl.ctypes.data_as(C.POINTER(C.c_int)),
            cnt.ctypes.data_as(C.POINTER(C.c_longlong)))
        if rc != 0:
            raise ValueError(f"oracle_forces failed ({rc})")
        out["force"][sl] = f; out["torque"][sl] = t; out["energy"][sl] = e
        out["fscale"][sl] = fs; out["tscale"][sl] = ts; out["flags"][sl] = fl
        out["virial"][r] = vir.reshape(3, 3); out["U"][r] = e.sum(); out["counts"][r] = cnt
    return out


def run(system, nsteps: int, dt: float, ensemble: str = "nve", kT: float = 1.0,
        tau: float = 0.5, par_eps: float = DEFAULT_PAR_EPS, thermo=None,
        P: float = 1.0, tau_P: float = 1.0):
    """Integrate ``nsteps`` from the system's state (copied, not modified).

    ensemble: "nve", "nvt" or "npt" (isotropic barostat at pressure P with
    barostat time tau_P; see oracle_run in dem_oracle.c).  thermo: per replica
    {xi, eta, p_e}.  Returns (state dict with pos, orient, vel, angmom, thermo
    (R, 3), box (R, dim) per replica, trace (R, nsteps, 5) = K_trans, K_rot, U,
    H, V per step).
    """
    lib = _load()
    dim = system.dim
    pk = pack_shapes(system.shapes)
    mass = np.array([sh["mass"] for sh in system.shapes], np.float64)
    inertia = np.zeros((len(system.shapes), 3))
    for s, sh in enumerate(system.shapes):
        I = np.asarray(sh["inertia"], np.float64).ravel()
        inertia[s, :len(I)] = I
    keep = []

    def dp(a):
        a, p = _d(a); keep.append(a); return p

    def ip(a):
        a, p = _i(a); keep.append(a); return p

    pos = np.array(system.pos, np.float64)
    orient = np.array(system.orient, np.float64)
    vel = np.array(system.vel, np.float64)
    angmom = np.array(system.angmom, np.float64)
    th = np.zeros((system.n_replicas, 3))
    if thermo is not None:
        t = np.atleast_2d(np.array(thermo, np.float64))
        th[:, :t.shape[1]] = t
    trace = np.zeros((system.n_replicas, nsteps, 5))
    boxes = np.array(system.box, np.float64).reshape(system.n_replicas, dim).copy()
    ens = {"nve": 0, "nvt": 1, "npt": 2}[ensemble]
    for r, sl in enumerate(system.replica_slices()):
        m = sl.stop - sl.start
        p_, o_, v_, a_ = (np.ascontiguousarray(x[sl]) for x in (pos, orient, vel, angmom))
        t_ = np.ascontiguousarray(th[r])
        b_ = np.ascontiguousarray(boxes[r])
        tr = np.zeros((nsteps, 5))
        rc = lib.oracle_run(dim, len(system.shapes), ip(pk["vert_off"]), dp(pk["verts"]),
                            ip(pk["shape_face_off"]), ip(pk["face_vert_off"]),
                            ip(pk["face_idx"]), dp(pk["rounding"]), dp(mass), dp(inertia),
                            float(system.epsilon), float(system.sigma), float(par_eps), m,
                            ip(system.shape_id[sl]),
                            p_.ctypes.data_as(C.POINTER(C.c_double)),
                            o_.ctypes.data_as(C.POINTER(C.c_double)),
                            v_.ctypes.data_as(C.POINTER(C.c_double)),
                            a_.ctypes.data_as(C.POINTER(C.c_double)),
                            b_.ctypes.data_as(C.POINTER(C.c_double)),
                            t_.ctypes.data_as(C.POINTER(C.c_double)),
                            int(nsteps), float(dt), ens, float(kT), float(tau), float(P),
                            float(tau_P), tr.ctypes.data_as(C.POINTER(C.c_double)))
        if rc != 0:
            raise ValueError(f"oracle_run failed ({rc})")
        pos[sl], orient[sl], vel[sl], angmom[sl] = p_, o_, v_, a_
        th[r] = t_
        boxes[r] = b_
        trace[r] = tr
    return dict(pos=pos, orient=orient, vel=vel, angmom=angmom, thermo=th, box=boxes), trace


def _vec(x):
    a = np.zeros(3)
    x = np.asarray(x, np.float64).ravel()
    a[:len(x)] = x
    return a


def point_segment(p, a, b):
    lib = _load()
    q = np.zeros(3)
    P, A, B = _vec(p), _vec(a), _vec(b)
    r = lib.oracle_point_segment(_d(P)[1], _d(A)[1], _d(B)[1], q.ctypes.data_as(C.POINTER(C.c_double)))
    return r, q


def point_face(p, poly):
    lib = _load()
    poly = np.ascontiguousarray(np.asarray(poly, np.float64).reshape(-1, 3))
    q = np.zeros(3)
    P = _vec(p)
    r = lib.oracle_point_face(_d(P)[1], len(poly), _d(poly)[1], q.ctypes.data_as(C.POINTER(C.c_double)))
    return r, q


def segment_segment(a1, b1, a2, b2, par_eps: float = DEFAULT_PAR_EPS):
    lib = _load()
    p1, p2 = np.zeros(3), np.zeros(3)
    par = C.c_int(0)
    v = [_vec(x) for x in (a1, b1, a2, b2)]
    r = lib.oracle_segment_segment(*[_d(x)[1] for x in v], float(par_eps),
                                   p1.ctypes.data_as(C.POINTER(C.c_double)),
                                   p2.ctypes.data_as(C.POINTER(C.c_double)), C.byref(par))
    return r, p1, p2, bool(par.value)


def wca(r, eps: float = 1.0, sigma: float = 1.0):
    """(U, -dU/dr) of the WCA potential at distance r."""
    lib = _load()
    f = C.c_double(0.0)
    u = lib.oracle_wca(float(r), float(eps), float(sigma), C.byref(f))
    return u, f.value


def set_parallel(threads: int = 1, cells: bool = False):
    """Timed CPU baseline only: evaluate forces with a cell-list pair search
    and/or OpenMP over particles (same pairs and terms; sums in another
    order).  set_parallel(1, False) restores the plain oracle the tests use.
    Per-particle scales and flags always come from the plain evaluation."""
    _load().oracle_set_parallel(int(threads), int(bool(cells)))


def max_threads() -> int:
    return int(_load().oracle_max_threads())
