"""Thin ctypes binding of libmpm.so (include/mpm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the CUDA kernels behind the
C-ABI.  If the compiled library is missing this module raises -- there is no
CPU fallback.  PyTorch is used only to find the current CUDA stream and to
hold device buffers for the device-pointer entry points.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmpm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mpm.h")

MPM_OK, MPM_ERR_ARG, MPM_ERR_OOM, MPM_ERR_CUDA = 0, -1, -2, -3
MPM_ERR_LEFT_MESH, MPM_ERR_NONFINITE, MPM_ERR_TIMEOUT, MPM_ERR_STATE = -4, -5, -6, -7
STATUS_NAMES = {0: "MPM_OK", -1: "MPM_ERR_ARG", -2: "MPM_ERR_OOM", -3: "MPM_ERR_CUDA",
                -4: "MPM_ERR_LEFT_MESH", -5: "MPM_ERR_NONFINITE", -6: "MPM_ERR_TIMEOUT", -7: "MPM_ERR_STATE"}
MPM_BC_FREE, MPM_BC_ROLLER, MPM_BC_FIXED, MPM_BC_FRICTION = 0, 1, 2, 3
MPM_USF, MPM_USL = 0, 1
MPM_FP64_PLAIN, MPM_FP32_MIXED = 0, 1
MPM_LINEAR_ELASTIC, MPM_MOHR_COULOMB, MPM_PLANE_STRESS_ELASTIC = 0, 1, 2


class MPMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mpm_mesh_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int32),
        ("ncells", C.c_int32 * 3),
        ("h", C.c_double),
        ("origin", C.c_double * 3),
        ("face_bc", C.c_int32 * 6),
        ("face_mu", C.c_double * 6),
        ("gravity", C.c_double * 3),
        ("dt", C.c_double),
        ("scheme", C.c_int32),
        ("precision", C.c_int32),
        ("mass_tol", C.c_double),
        ("stream", C.c_void_p),
    ]


class mpm_material(C.Structure):
    _fields_ = [
        ("model", C.c_int32),
        ("E", C.c_double),
        ("nu", C.c_double),
        ("rho", C.c_double),
        ("phi", C.c_double),
        ("c", C.c_double),
        ("psi", C.c_double),
    ]


_lock = threading.Lock()
_lib = None


def load():
    """Load libmpm.so (building it first when nvcc is present and the
    library is missing or stale).  Raises if it cannot be had."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _b
        try:
            _b.build()
        except RuntimeError as e:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libmpm.so is missing and cannot be built: {e}") from e
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmpm.so not found at {LIB_PATH}")
        L = C.CDLL(LIB_PATH)
        vp, dp, i32p, i64p, u32p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), \
            C.POINTER(C.c_int64), C.POINTER(C.c_uint32)
        sig = {
            "mpm_create_mesh": [C.POINTER(mpm_mesh_desc), C.POINTER(vp)],
            "mpm_add_particles": [vp, C.c_int64, dp, dp, dp, C.POINTER(mpm_material), dp, dp, i64p],
            "mpm_step": [vp, C.c_int64],
            "mpm_sync": [vp],
            "mpm_num_particles": [vp, i64p],
            "mpm_read_particles": [vp, dp, dp, dp, dp, dp, dp, i64p],
            "mpm_conservation": [vp, dp],
            "mpm_read_binning": [vp, i32p, i32p, i32p],
            "mpm_destroy": [vp],
            "mpm_sort_keys": [vp, vp, C.c_int64, C.c_int32, vp],
            "mpm_sort_keys_static": [vp, vp, C.c_int64, C.c_int32, vp],
            "mpm_footprint": [C.POINTER(mpm_mesh_desc), C.c_int64, C.c_int32, i64p],
            "mpm_batch_create": [C.c_int64, C.c_int32, vp, C.POINTER(vp)],
            "mpm_batch_admit": [vp, vp, i32p],
            "mpm_batch_room": [vp, i64p, i32p],
            "mpm_batch_evict": [vp, C.c_int32],
            "mpm_batch_step": [vp, C.c_int64],
            "mpm_batch_poll": [vp, C.c_int32, i32p, i64p],
            "mpm_batch_step_kernels": [vp, i32p],
            "mpm_batch_destroy": [vp],
            "mpm_step_kernels": [vp, i32p],
            "mpm_set_scan_fault": [vp, C.c_int32, C.c_int32],
            "mpm_set_loads": [vp, dp, C.c_double],
            "mpm_set_node_coordinates": [vp, dp],
            "mpm_set_face_stress": [vp, dp],
            "mpm_material_update": [C.POINTER(mpm_material), C.c_int32, C.c_int64, dp, dp, dp, dp, dp, vp],
            "mpm_set_phase_timing": [vp, C.c_int32],
            "mpm_phase_times": [vp, C.POINTER(C.c_float), i32p],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.mpm_last_error.argtypes = [vp]
        L.mpm_last_error.restype = C.c_char_p
        _lib = L
        return L


def header_entry_points():
    """Names of the functions include/mpm.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:mpm_status|const char \*)\s*(mpm_\w+)\s*\(", txt, re.M)))


def _check(h, st: int, what: str):
    if st != MPM_OK:
        msg = load().mpm_last_error(h).decode() if h else what
        raise MPMError(st, f"{what}: {msg}")


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def current_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream or None)


def make_desc(dim, ncells, h, origin=(0, 0, 0), face_bc=(0,) * 6, face_mu=(0,) * 6, gravity=(0, 0, 0),
              dt=1e-5, scheme=MPM_USL, precision=MPM_FP32_MIXED, mass_tol=1e-12, stream=None):
    d = mpm_mesh_desc()
    d.dim = int(dim)
    nc = list(ncells) + [1] * (3 - len(ncells))
    for k in range(3):
        d.ncells[k] = int(nc[k])
        d.origin[k] = float(origin[k])
        d.gravity[k] = float(gravity[k])
    for f in range(6):
        d.face_bc[f] = int(face_bc[f])
        d.face_mu[f] = float(face_mu[f])
    d.h, d.dt, d.scheme, d.precision, d.mass_tol = float(h), float(dt), int(scheme), int(precision), float(mass_tol)
    d.stream = stream
    return d


def make_material(model=MPM_LINEAR_ELASTIC, E=1e7, nu=0.3, rho=1000.0, phi=0.0, c=0.0, psi=0.0):
    m = mpm_material()
    m.model, m.E, m.nu, m.rho, m.phi, m.c, m.psi = int(model), E, nu, rho, phi, c, psi
    return m


# ---- the C entry points, one Python function each --------------------------

def mpm_create_mesh(desc: mpm_mesh_desc):
    h = C.c_void_p()
    st = load().mpm_create_mesh(C.byref(desc), C.byref(h))
    _check(None, st, "mpm_create_mesh")
    return h


def mpm_add_particles(h, pos, vel, vol, mat: mpm_material, cohesion=None, stress0=None) -> int:
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    vol = np.ascontiguousarray(vol, np.float64)
    coh = None if cohesion is None else np.ascontiguousarray(cohesion, np.float64)
    s0 = None if stress0 is None else np.ascontiguousarray(stress0, np.float64)
    first = C.c_int64()
    st = load().mpm_add_particles(h, pos.shape[0], _dp(pos), _dp(vel), _dp(vol), C.byref(mat), _dp(coh),
                                  _dp(s0), C.byref(first))
    _check(h, st, "mpm_add_particles")
    return first.value


def mpm_step(h, nsteps: int):
    _check(h, load().mpm_step(h, int(nsteps)), "mpm_step")


def mpm_sync(h) -> int:
    """Wait for the stream; returns the latched status (raises on CUDA errors)."""
    st = load().mpm_sync(h)
    if st in (MPM_ERR_CUDA, MPM_ERR_OOM):
        _check(h, st, "mpm_sync")
    return st


def mpm_num_particles(h) -> int:
    n = C.c_int64()
    _check(h, load().mpm_num_particles(h, C.byref(n)), "mpm_num_particles")
    return n.value


def mpm_read_particles(h, dim: int, fields=("pos", "vel", "stress", "strain", "vol", "epsp", "cell"), out=None):
    """Particle state in insertion order; returns (dict, status).  `out` may
    supply the destination arrays (C-contiguous, float64 -- int64 for
    "cell" -- of the field's shape), e.g. views of pinned host memory."""
    n = mpm_num_particles(h)
    given = out or {}
    out = {}
    shapes = {"pos": (n, dim), "vel": (n, dim), "stress": (n, 6), "strain": (n, 6), "vol": (n,), "epsp": (n,),
              "cell": (n,)}
    for k, s in shapes.items():
        dt = np.int64 if k == "cell" else np.float64
        if k not in fields:
            out[k] = None
        elif k in given:
            a = given[k]
            if a.shape != s or a.dtype != dt or not a.flags.c_contiguous:
                raise MPMError(MPM_ERR_ARG, f"mpm_read_particles: out[{k!r}] must be C-contiguous {dt.__name__} {s}")
            out[k] = a
        else:
            out[k] = np.empty(s, dt)
    cptr = None if out["cell"] is None else out["cell"].ctypes.data_as(C.POINTER(C.c_int64))
    st = load().mpm_read_particles(h, _dp(out["pos"]), _dp(out["vel"]), _dp(out["stress"]), _dp(out["strain"]),
                                   _dp(out["vol"]), _dp(out["epsp"]), cptr)
    if st in (MPM_ERR_CUDA, MPM_ERR_OOM, MPM_ERR_ARG):
        _check(h, st, "mpm_read_particles")
    return {k: v for k, v in out.items() if v is not None}, st


def mpm_conservation(h):
    out = np.zeros(8)
    st = load().mpm_conservation(h, _dp(out))
    if st in (MPM_ERR_CUDA, MPM_ERR_OOM, MPM_ERR_ARG):
        _check(h, st, "mpm_conservation")
    return {"mass": out[0], "momentum": out[1:4].copy(), "ke": out[4], "se": out[5], "alive": int(out[6]),
            "volume": out[7]}, st


def mpm_read_binning(h):
    n = mpm_num_particles(h)
    key = np.empty(n, np.int32)
    perm = np.empty(n, np.int32)
    td = np.zeros(3, np.int32)
    st = load().mpm_read_binning(h, key.ctypes.data_as(C.POINTER(C.c_int32)),
                                 perm.ctypes.data_as(C.POINTER(C.c_int32)), td.ctypes.data_as(C.POINTER(C.c_int32)))
    if st in (MPM_ERR_CUDA, MPM_ERR_OOM, MPM_ERR_ARG, MPM_ERR_STATE):
        _check(h, st, "mpm_read_binning")
    return key, perm, tuple(int(t) for t in td)


def mpm_set_phase_timing(h, enable: bool):
    _check(h, load().mpm_set_phase_timing(h, int(bool(enable))), "mpm_set_phase_timing")


def mpm_phase_times(h):
    """Durations (ms) of the last step's phases."""
    ms = (C.c_float * 8)()
    n = C.c_int32()
    _check(h, load().mpm_phase_times(h, ms, C.byref(n)), "mpm_phase_times")
    return [float(ms[i]) for i in range(n.value)]


def mpm_destroy(h):
    load().mpm_destroy(h)


def mpm_last_error(h) -> str:
    return load().mpm_last_error(h).decode()


def mpm_sort_keys(d_keys, d_perm, n: int, key_bits: int, stream=None):
    """Device pointers (ints or torch tensors' data_ptr())."""
    kp = d_keys.data_ptr() if hasattr(d_keys, "data_ptr") else int(d_keys)
    pp = d_perm.data_ptr() if hasattr(d_perm, "data_ptr") else int(d_perm)
    st = load().mpm_sort_keys(C.c_void_p(kp), C.c_void_p(pp), int(n), int(key_bits),
                              stream if stream is not None else current_stream())
    _check(None, st, "mpm_sort_keys")


MPM_SORT_STATIC_MAX_KEYS = 1 << 20


def mpm_sort_keys_static(d_keys, d_perm, n: int, key_bits: int, stream=None):
    """The sort without any device allocation (fixed library scratch, at most
    MPM_SORT_STATIC_MAX_KEYS keys).  Only enqueues on the stream: synchronise
    before reading d_perm."""
    kp = d_keys.data_ptr() if hasattr(d_keys, "data_ptr") else int(d_keys)
    pp = d_perm.data_ptr() if hasattr(d_perm, "data_ptr") else int(d_perm)
    st = load().mpm_sort_keys_static(C.c_void_p(kp), C.c_void_p(pp), int(n), int(key_bits),
                                     stream if stream is not None else current_stream())
    _check(None, st, "mpm_sort_keys_static")


def mpm_footprint(desc: mpm_mesh_desc, n: int, has_cohesion: bool = False) -> int:
    out = C.c_int64()
    _check(None, load().mpm_footprint(C.byref(desc), int(n), int(bool(has_cohesion)), C.byref(out)), "mpm_footprint")
    return out.value


def mpm_batch_create(stream=None, hbm_budget_bytes: int = 0, max_slots: int = 1 << 20):
    b = C.c_void_p()
    _check(None, load().mpm_batch_create(int(hbm_budget_bytes), int(max_slots), stream, C.byref(b)),
           "mpm_batch_create")
    return b


def mpm_batch_admit(b, h) -> int:
    """Slot of the admitted mesh; raises MPMError(MPM_ERR_OOM) when the batch
    has no free slot or not enough of its memory budget left."""
    slot = C.c_int32()
    st = load().mpm_batch_admit(b, h, C.byref(slot))
    _check(h, st, "mpm_batch_admit")
    return slot.value


def mpm_batch_room(b):
    """(bytes left in the batch's budget, free slots)."""
    fb, fs = C.c_int64(), C.c_int32()
    _check(None, load().mpm_batch_room(b, C.byref(fb), C.byref(fs)), "mpm_batch_room")
    return fb.value, fs.value


def mpm_batch_step_kernels(b) -> int:
    k = C.c_int32()
    _check(None, load().mpm_batch_step_kernels(b, C.byref(k)), "mpm_batch_step_kernels")
    return k.value


def mpm_set_loads(h, face_traction=None, damping: float = 0.0):
    """face_traction: 6 x 3 tractions (faces -x,+x,-y,+y,-z,+z) or None."""
    t = None if face_traction is None else np.ascontiguousarray(face_traction, np.float64).reshape(18)
    _check(h, load().mpm_set_loads(h, _dp(t), float(damping)), "mpm_set_loads")


def mpm_set_node_coordinates(h, node_xyz):
    """node_xyz: (nodes, dim) coordinates of a mapped mesh's nodes, x fastest."""
    X = np.ascontiguousarray(node_xyz, np.float64)
    _check(h, load().mpm_set_node_coordinates(h, _dp(X)), "mpm_set_node_coordinates")


def mpm_set_face_stress(h, face_stress=None):
    """face_stress: 6 x 6 (faces -x,+x,-y,+y,-z,+z; Voigt xx yy zz xy yz xz) or None."""
    S = None if face_stress is None else np.ascontiguousarray(face_stress, np.float64).reshape(36)
    _check(h, load().mpm_set_face_stress(h, _dp(S)), "mpm_set_face_stress")


def mpm_set_scan_fault(h, withhold_chunk: int, spin_limit: int = 1 << 20):
    _check(h, load().mpm_set_scan_fault(h, int(withhold_chunk), int(spin_limit)), "mpm_set_scan_fault")


def mpm_step_kernels(h) -> int:
    k = C.c_int32()
    _check(h, load().mpm_step_kernels(h, C.byref(k)), "mpm_step_kernels")
    return k.value


def mpm_batch_evict(b, slot: int):
    _check(None, load().mpm_batch_evict(b, int(slot)), "mpm_batch_evict")


def mpm_batch_step(b, nsteps: int):
    _check(None, load().mpm_batch_step(b, int(nsteps)), "mpm_batch_step")


def mpm_batch_poll(b, nslots: int, with_steps: bool = False):
    """Per-slot status (and, with_steps, the batched steps each slot's mesh
    has taken since its admission, -1 for an empty slot)."""
    out = (C.c_int32 * max(1, nslots))()
    steps = (C.c_int64 * max(1, nslots))()
    _check(None, load().mpm_batch_poll(b, int(nslots), out, steps), "mpm_batch_poll")
    status = [int(out[i]) for i in range(nslots)]
    if with_steps:
        return status, [int(steps[i]) for i in range(nslots)]
    return status


def mpm_batch_destroy(b):
    load().mpm_batch_destroy(b)


def mpm_material_update(mat: mpm_material, precision: int, sig, deps, cohesion=None, stream=None):
    sig = np.ascontiguousarray(sig, np.float64).reshape(-1, 6)
    deps = np.ascontiguousarray(deps, np.float64).reshape(-1, 6)
    coh = None if cohesion is None else np.ascontiguousarray(cohesion, np.float64)
    n = sig.shape[0]
    out = np.empty((n, 6))
    dep = np.empty(n)
    st = load().mpm_material_update(C.byref(mat), int(precision), n, _dp(sig), _dp(deps), _dp(coh), _dp(out),
                                    _dp(dep), stream if stream is not None else current_stream())
    _check(None, st, "mpm_material_update")
    return out, dep


# ---- convenience -----------------------------------------------------------

class Simulation:
    """One mesh handle built from a workload description (see workloads.py)."""

    def __init__(self, wl, precision=None, scheme=None, stream=None, mass_tol=1e-12, stress0=None):
        """stress0: optional (n, 6) initial stresses (Voigt xx yy zz xy yz xz; zeros if None)."""
        self.wl = wl
        self.dim = wl.dim
        self.precision = wl.precision if precision is None else precision
        self.scheme = wl.scheme if scheme is None else scheme
        if stream is None:
            stream = current_stream()
        self.desc = make_desc(wl.dim, wl.ncells, wl.h, wl.origin, wl.face_bc, wl.face_mu, wl.gravity, wl.dt,
                              self.scheme, self.precision, mass_tol, stream)
        self.mat = make_material(**wl.material)
        self.h = mpm_create_mesh(self.desc)
        try:
            X = getattr(wl, "node_xyz", None)
            if X is not None:
                mpm_set_node_coordinates(self.h, np.asarray(X)[:, : wl.dim])
            if wl.n:
                mpm_add_particles(self.h, wl.pos, wl.vel, wl.vol, self.mat, wl.coh, stress0)
            trac = getattr(wl, "face_traction", None)
            damp = float(getattr(wl, "damping", 0.0))
            if damp > 0.0 or (trac is not None and np.any(np.asarray(trac) != 0.0)):
                mpm_set_loads(self.h, trac, damp)
            fs = getattr(wl, "face_stress", None)
            if fs is not None and np.any(np.asarray(fs) != 0.0):
                mpm_set_face_stress(self.h, fs)
        except Exception:
            mpm_destroy(self.h)
            raise

    def step(self, n=1):
        mpm_step(self.h, n)

    def sync(self):
        return mpm_sync(self.h)

    def read(self, fields=("pos", "vel", "stress", "strain", "vol", "epsp", "cell"), out=None):
        return mpm_read_particles(self.h, self.dim, fields, out)

    def conservation(self):
        return mpm_conservation(self.h)

    def binning(self):
        return mpm_read_binning(self.h)

    def close(self):
        if self.h:
            mpm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
