"""ctypes binding of libdem (include/dem.h): the same entry points, argument
marshalling only.  Every step of the computation runs in the CUDA library;
there is no Python or CPU fallback: if libdem.so is missing or fails to load,
every call raises.

Arrays may be numpy arrays (host) or CUDA torch tensors (device, passed with
device_ptrs=1, used on the context's stream).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdem.so")

DEM_OK = 0
DEM_ERR_ARG = -1
DEM_ERR_CUDA = -2
DEM_ERR_NONFINITE = -3
DEM_ERR_NLIST_OVERFLOW = -4
DEM_ERR_TIMEOUT = -5
DEM_ERR_BOX = -6
DEM_ERR_STATE = -7
DEM_ERR_NOMEM = -8

DEM_FP64, DEM_FP32, DEM_FP32_COMP = 0, 1, 2
DEM_NVE, DEM_NVT, DEM_NPT = 0, 1, 2
DEM_DECOMP_AUTO, DEM_DECOMP_THREAD, DEM_DECOMP_WARP, DEM_DECOMP_STAGED, DEM_DECOMP_SPLIT = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": DEM_FP64, "fp32": DEM_FP32, "fp32c": DEM_FP32_COMP}

# Every symbol include/dem.h declares (checked by the CPU tests).
EXPORTS = ["dem_create", "dem_set_state", "dem_get_state", "dem_set_thermostat", "dem_step",
           "dem_compute", "dem_get_forces", "dem_get_energy", "dem_get_particle_energy",
           "dem_get_virial", "dem_set_box", "dem_set_param", "dem_get_param", "dem_autotune",
           "dem_get_counters", "dem_set_stream", "dem_shape_info", "dem_last_error",
           "dem_destroy", "dem_forces_noalloc", "dem_set_barostat", "dem_get_box",
           "dem_fma_peak", "dem_check_conversions"]
DEM_NOALLOC_MAX_N = 16384
DEM_NOALLOC_MAX_NEIGHBOURS = 64


class DemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdem error {code}: {msg}")
        self.code = code


class dem_shape(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_verts", C.c_int), ("verts", C.POINTER(C.c_double)),
                ("n_faces", C.c_int), ("face_offsets", C.POINTER(C.c_int)),
                ("face_verts", C.POINTER(C.c_int)), ("rounding_radius", C.c_double),
                ("mass", C.c_double), ("inertia", C.POINTER(C.c_double))]


_lib = None


def load():
    """Load libdem.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libdem.so not found at {LIB_PATH}; build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    vp, dp, ip, lp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_longlong)
    sig = {
        "dem_create": [C.POINTER(vp), C.POINTER(dem_shape), C.c_int, C.c_double, C.c_double, dp,
                       C.c_int, ip, C.c_int],
        "dem_set_state": [vp, vp, vp, vp, vp, vp, C.c_int],
        "dem_get_state": [vp, vp, vp, vp, vp, vp, C.c_int],
        "dem_set_thermostat": [vp, dp],
        "dem_set_barostat": [vp, C.c_double, C.c_double],
        "dem_get_box": [vp, dp],
        "dem_step": [vp, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double],
        "dem_compute": [vp],
        "dem_get_forces": [vp, vp, vp, C.c_int],
        "dem_get_energy": [vp, dp, dp, dp],
        "dem_get_particle_energy": [vp, vp, C.c_int],
        "dem_get_virial": [vp, dp],
        "dem_set_box": [vp, dp],
        "dem_set_param": [vp, C.c_char_p, C.c_double],
        "dem_get_param": [vp, C.c_char_p, dp],
        "dem_autotune": [vp],
        "dem_get_counters": [vp, lp],
        "dem_set_stream": [vp, vp],
        "dem_shape_info": [C.POINTER(dem_shape), dp],
        "dem_destroy": [vp],
        "dem_forces_noalloc": [C.POINTER(dem_shape), C.c_int, C.c_double, C.c_double, dp,
                               C.c_int, vp, vp, vp, C.c_int, vp, vp, vp, vp],
        "dem_fma_peak": [C.c_int, C.c_int, dp, dp],
        "dem_check_conversions": [C.c_ulonglong, C.c_ulonglong, C.POINTER(C.c_ulonglong)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None if name == "dem_destroy" else C.c_int
    lib.dem_last_error.argtypes = [vp]
    lib.dem_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc, ctx=None):
    if rc != DEM_OK:
        msg = load().dem_last_error(ctx)
        raise DemError(rc, msg.decode() if msg else "")
    return rc


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    """Pointer of a host numpy array or a CUDA torch tensor (None stays None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def make_shape(shape: dict):
    """dem_shape from a shape dict (keys dim, verts, faces, rounding, mass,
    inertia); returns (struct, keep-alive list)."""
    dim = int(shape["dim"])
    verts = _host(np.asarray(shape["verts"], np.float64).reshape(-1, dim), np.float64)
    keep = [verts]
    faces = shape.get("faces") or []
    offs = _host(np.cumsum([0] + [len(f) for f in faces]), np.int32)
    fv = _host([k for f in faces for k in f] or [0], np.int32)
    keep += [offs, fv]
    inertia = shape.get("inertia")
    inert_p = None
    if inertia is not None:
        ia = _host(np.asarray(inertia, np.float64).ravel(), np.float64)
        keep.append(ia)
        inert_p = ia.ctypes.data_as(C.POINTER(C.c_double))
    s = dem_shape(dim, len(verts), verts.ctypes.data_as(C.POINTER(C.c_double)), len(faces),
                  offs.ctypes.data_as(C.POINTER(C.c_int)), fv.ctypes.data_as(C.POINTER(C.c_int)),
                  float(shape["rounding"]), float(shape.get("mass", 1.0)), inert_p)
    return s, keep


def dem_shape_info(shape: dict) -> np.ndarray:
    """Host-only derived shape properties (see dem.h)."""
    lib = load()
    s, keep = make_shape(shape)
    out = np.zeros(8)
    _check(lib.dem_shape_info(C.byref(s), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out[:7]


def dem_create(shapes: Sequence[dict], epsilon: float, sigma: float, box, replica_sizes,
               precision: int):
    lib = load()
    arr = (dem_shape * len(shapes))()
    keep = []
    for k, sh in enumerate(shapes):
        s, kk = make_shape(sh)
        arr[k] = s
        keep += kk
    dim = int(shapes[0]["dim"])
    box = _host(np.asarray(box, np.float64).reshape(-1, dim), np.float64)
    sizes = _host(replica_sizes, np.int32)
    ctx = C.c_void_p()
    rc = lib.dem_create(C.byref(ctx), arr, len(shapes), float(epsilon), float(sigma),
                        box.ctypes.data_as(C.POINTER(C.c_double)), len(sizes),
                        sizes.ctypes.data_as(C.POINTER(C.c_int)), int(precision))
    _check(rc, None)
    return ctx


def dem_set_state(ctx, shape_id, pos, orient, vel, angmom, device_ptrs: int = 0):
    lib = load()
    arrays = (shape_id, pos, orient, vel, angmom)
    if device_ptrs or all(hasattr(a, "data_ptr") for a in arrays):
        # CUDA tensors (device_ptrs=1), or host torch tensors (e.g. pinned
        # memory) passed as they are: int32 / float64, contiguous
        return _check(lib.dem_set_state(ctx, *[_ptr(a) for a in arrays], int(device_ptrs)), ctx)
    arrs = [_host(shape_id, np.int32)] + [_host(a, np.float64) for a in (pos, orient, vel, angmom)]
    return _check(lib.dem_set_state(ctx, *[_ptr(a) for a in arrs], 0), ctx)


def dem_get_state(ctx, pos=None, orient=None, vel=None, angmom=None, thermostat=None,
                  device_ptrs: int = 0):
    lib = load()
    return _check(lib.dem_get_state(ctx, _ptr(pos), _ptr(orient), _ptr(vel), _ptr(angmom),
                                    _ptr(thermostat), int(device_ptrs)), ctx)


def dem_set_thermostat(ctx, thermostat):
    """Per replica (xi, eta, p_e)."""
    lib = load()
    t = _host(thermostat, np.float64)
    return _check(lib.dem_set_thermostat(ctx, t.ctypes.data_as(C.POINTER(C.c_double))), ctx)


def dem_set_barostat(ctx, P: float, tau_P: float):
    lib = load()
    return _check(lib.dem_set_barostat(ctx, float(P), float(tau_P)), ctx)


def dem_get_box(ctx, n_replicas: int, dim: int) -> np.ndarray:
    lib = load()
    out = np.zeros((n_replicas, dim))
    _check(lib.dem_get_box(ctx, out.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return out


def dem_step(ctx, n: int, dt: float, ensemble: int, kT: float = 1.0, tau_T: float = 1.0):
    return _check(load().dem_step(ctx, int(n), float(dt), int(ensemble), float(kT),
                                  float(tau_T)), ctx)


def dem_compute(ctx):
    return _check(load().dem_compute(ctx), ctx)


def dem_get_forces(ctx, force=None, torque=None, device_ptrs: int = 0):
    return _check(load().dem_get_forces(ctx, _ptr(force), _ptr(torque), int(device_ptrs)), ctx)


def dem_get_energy(ctx, n_replicas: int):
    U, K, H = np.zeros(n_replicas), np.zeros(n_replicas), np.zeros(n_replicas)
    dp = C.POINTER(C.c_double)
    _check(load().dem_get_energy(ctx, U.ctypes.data_as(dp), K.ctypes.data_as(dp),
                                 H.ctypes.data_as(dp)), ctx)
    return U, K, H


def dem_get_particle_energy(ctx, out, device_ptrs: int = 0):
    return _check(load().dem_get_particle_energy(ctx, _ptr(out), int(device_ptrs)), ctx)


def dem_get_virial(ctx, n_replicas: int):
    W = np.zeros((n_replicas, 6))
    _check(load().dem_get_virial(ctx, W.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return W


def dem_set_box(ctx, box):
    b = _host(box, np.float64)
    return _check(load().dem_set_box(ctx, b.ctypes.data_as(C.POINTER(C.c_double))), ctx)


def dem_set_param(ctx, name: str, value: float):
    return _check(load().dem_set_param(ctx, name.encode(), float(value)), ctx)


def dem_get_param(ctx, name: str) -> float:
    v = C.c_double(0.0)
    _check(load().dem_get_param(ctx, name.encode(), C.byref(v)), ctx)
    return v.value


def dem_autotune(ctx):
    return _check(load().dem_autotune(ctx), ctx)


def dem_get_counters(ctx) -> np.ndarray:
    c = np.zeros(20, np.int64)
    _check(load().dem_get_counters(ctx, c.ctypes.data_as(C.POINTER(C.c_longlong))), ctx)
    return c


def dem_set_stream(ctx, stream_handle: Optional[int]):
    return _check(load().dem_set_stream(ctx, C.c_void_p(stream_handle) if stream_handle else None),
                  ctx)


def dem_destroy(ctx):
    if ctx:
        load().dem_destroy(ctx)


def dem_fma_peak(precision: int, iters: int):
    """Measured FMA throughput (TFLOP/s, ms of the timed launch) of the
    current device in FP32 (DEM_FP32) or FP64 (DEM_FP64)."""
    t, ms = C.c_double(0.0), C.c_double(0.0)
    _check(load().dem_fma_peak(int(precision), int(iters), C.byref(t), C.byref(ms)))
    return t.value, ms.value


def dem_check_conversions(n: int, seed: int = 1607_02427):
    """Mismatches (double to float, float to double) of the integrator's
    integer-operation conversions against the conversion instructions over n
    hashed inputs."""
    out = (C.c_ulonglong * 2)()
    _check(load().dem_check_conversions(C.c_ulonglong(int(n)), C.c_ulonglong(int(seed)), out))
    return int(out[0]), int(out[1])


def dem_forces_noalloc(shapes: Sequence[dict], epsilon: float, sigma: float, box, shape_id,
                       pos, orient, precision: int, force, torque, energy=None,
                       stream_handle: Optional[int] = None):
    """Forces of one system with no device allocation (see dem.h).  shape_id,
    pos, orient, force, torque and energy are CUDA tensors: contiguous,
    int32 (shape_id) or float64 (the rest), with the sizes dem.h states;
    anything else raises ValueError before the library is called (the
    library cannot check device arrays it is handed)."""
    import torch
    lib = load()
    if not isinstance(shape_id, torch.Tensor) or shape_id.dim() != 1:
        raise ValueError("shape_id must be a 1-D CUDA tensor")
    n = int(shape_id.shape[0])
    dim = int(shapes[0]["dim"])
    widths = {"pos": dim, "orient": 4 if dim == 3 else 1, "force": dim,
              "torque": 3 if dim == 3 else 1, "energy": 1}
    named = {"shape_id": (shape_id, torch.int32, 1), "pos": (pos, torch.float64, widths["pos"]),
             "orient": (orient, torch.float64, widths["orient"]),
             "force": (force, torch.float64, widths["force"]),
             "torque": (torque, torch.float64, widths["torque"])}
    if energy is not None:
        named["energy"] = (energy, torch.float64, 1)
    for nm, (t, dt, w) in named.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{nm} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{nm} must have dtype {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{nm} must be contiguous")
        if t.numel() != n * w:
            raise ValueError(f"{nm} must hold {n} x {w} values, got {t.numel()}")
    arr = (dem_shape * len(shapes))()
    keep = []
    for k, sh in enumerate(shapes):
        s, kk = make_shape(sh)
        arr[k] = s
        keep += kk
    b = _host(np.asarray(box, np.float64).ravel(), np.float64)
    return _check(lib.dem_forces_noalloc(arr, len(shapes), float(epsilon), float(sigma),
                                         b.ctypes.data_as(C.POINTER(C.c_double)), n,
                                         _ptr(shape_id), _ptr(pos), _ptr(orient), int(precision),
                                         _ptr(force), _ptr(torque), _ptr(energy),
                                         C.c_void_p(stream_handle) if stream_handle else None))


class DEM:
    """Owner of one context: a batch of replica systems (see workloads.System)."""

    def __init__(self, system, precision: int = DEM_FP32_COMP, **params):
        self.dim = system.dim
        self.n = system.n
        self.n_replicas = system.n_replicas
        self.ctx = dem_create(system.shapes, system.epsilon, system.sigma, system.box,
                              system.replica_sizes, precision)
        try:
            for k, v in params.items():
                dem_set_param(self.ctx, k, v)
            dem_set_state(self.ctx, system.shape_id, system.pos, system.orient, system.vel,
                          system.angmom)
        except Exception:
            self.close()
            raise

    def close(self):
        if getattr(self, "ctx", None):
            dem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # convenience wrappers returning numpy arrays
    def forces(self):
        f = np.zeros((self.n, self.dim))
        t = np.zeros((self.n, 3 if self.dim == 3 else 1))
        dem_get_forces(self.ctx, f, t)
        return f, t

    def particle_energy(self):
        e = np.zeros(self.n)
        dem_get_particle_energy(self.ctx, e)
        return e

    def energy(self):
        return dem_get_energy(self.ctx, self.n_replicas)

    def virial(self):
        return dem_get_virial(self.ctx, self.n_replicas)

    def state(self):
        pos = np.zeros((self.n, self.dim))
        orient = np.zeros((self.n, 4 if self.dim == 3 else 1))
        vel = np.zeros((self.n, self.dim))
        ang = np.zeros((self.n, 3 if self.dim == 3 else 1))
        th = np.zeros((self.n_replicas, 3))
        dem_get_state(self.ctx, pos, orient, vel, ang, th)
        return dict(pos=pos, orient=orient, vel=vel, angmom=ang, thermo=th,
                    box=dem_get_box(self.ctx, self.n_replicas, self.dim))

    def step(self, n, dt, ensemble=DEM_NVE, kT=1.0, tau_T=0.5):
        dem_step(self.ctx, n, dt, ensemble, kT, tau_T)

    def compute(self):
        dem_compute(self.ctx)

    def counters(self):
        return dem_get_counters(self.ctx)

    def set_param(self, name, value):
        dem_set_param(self.ctx, name, value)

    def get_param(self, name):
        return dem_get_param(self.ctx, name)

    def set_box(self, box):
        dem_set_box(self.ctx, box)

    def set_barostat(self, P, tau_P):
        dem_set_barostat(self.ctx, P, tau_P)

    def box(self):
        return dem_get_box(self.ctx, self.n_replicas, self.dim)

    def set_thermostat(self, th):
        dem_set_thermostat(self.ctx, th)
