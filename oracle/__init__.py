"""FP64 CPU oracle for the explicit material point method step.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` are the only callers.  The
product library (``paper_1909_13380_gb300``) never imports this package and
shares no code with it.

The arithmetic lives in ``mpm_oracle.c`` (plain C, FP64, single thread); this
module only compiles it with gcc and marshals numpy arrays through ctypes.
Citations of the paper's passages are in the C file next to each function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libmpm_oracle.so")

OK, ARG, LEFT_MESH, NONFINITE = 0, -1, -4, -5
BC_FREE, BC_ROLLER, BC_FIXED, BC_FRICTION = 0, 1, 2, 3
USF, USL = 0, 1
LINEAR_ELASTIC, MOHR_COULOMB, PLANE_STRESS_ELASTIC = 0, 1, 2


class _Mesh(C.Structure):
    _fields_ = [
        ("dim", C.c_int32),
        ("n", C.c_int32 * 3),
        ("h", C.c_double),
        ("origin", C.c_double * 3),
        ("face_bc", C.c_int32 * 6),
        ("face_mu", C.c_double * 6),
        ("g", C.c_double * 3),
        ("dt", C.c_double),
        ("scheme", C.c_int32),
        ("mass_tol", C.c_double),
        ("face_traction", (C.c_double * 3) * 6),
        ("damping", C.c_double),
        ("face_stress", (C.c_double * 6) * 6),
    ]


class _Material(C.Structure):
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


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (no FMA contraction so
    that x86 and Arm hosts round identically)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            L.oracle_num_nodes.restype = C.c_int64
            L.oracle_num_nodes.argtypes = [C.POINTER(_Mesh)]
            L.oracle_work_size.restype = C.c_int64
            L.oracle_work_size.argtypes = [C.POINTER(_Mesh)]
            L.oracle_locate.restype = C.c_int
            L.oracle_locate.argtypes = [C.POINTER(_Mesh), dp, ip, dp]
            L.oracle_shape.restype = None
            L.oracle_shape.argtypes = [C.c_int32, dp, dp, dp]
            L.oracle_p2g.restype = None
            L.oracle_p2g.argtypes = [C.POINTER(_Mesh), C.c_int64, dp, dp, dp, dp, dp, ip, dp, dp, dp]
            L.oracle_constrain_node.restype = None
            L.oracle_constrain_node.argtypes = [C.POINTER(_Mesh), ip, dp, dp, dp]
            L.oracle_eig_sym3.restype = None
            L.oracle_eig_sym3.argtypes = [dp, dp, dp]
            L.oracle_mc_return.restype = C.c_int
            L.oracle_mc_return.argtypes = [C.c_double] * 5 + [dp, dp, dp]
            L.oracle_stress_update.restype = None
            L.oracle_stress_update.argtypes = [C.POINTER(_Material), C.c_double, dp, dp, dp]
            L.oracle_step.restype = C.c_int
            L.oracle_step.argtypes = [C.POINTER(_Mesh), C.POINTER(_Material), C.c_int64,
                                      dp, dp, dp, dp, dp, dp, dp, dp, ip, dp, C.c_int64]
            L.oracle_iso_natural.restype = C.c_int
            L.oracle_iso_natural.argtypes = [C.POINTER(_Mesh), dp, ip, dp, dp]
            L.oracle_iso_locate.restype = C.c_int
            L.oracle_iso_locate.argtypes = [C.POINTER(_Mesh), dp, dp, ip, dp]
            L.oracle_iso_basis.restype = None
            L.oracle_iso_basis.argtypes = [C.POINTER(_Mesh), dp, ip, dp, dp, dp]
            L.oracle_face_normal.restype = None
            L.oracle_face_normal.argtypes = [C.POINTER(_Mesh), dp, C.c_int32, ip, dp]
            L.oracle_step_mapped.restype = C.c_int
            L.oracle_step_mapped.argtypes = [C.POINTER(_Mesh), dp, C.POINTER(_Material), C.c_int64,
                                             dp, dp, dp, dp, dp, dp, dp, dp, ip, ip, dp, C.c_int64]
            L.oracle_conservation.restype = None
            L.oracle_conservation.argtypes = [C.c_int64, dp, dp, dp, dp, dp, ip, dp]
            _lib = L
        return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


@dataclass
class Mesh:
    """Background mesh and step parameters (oracle's own description)."""
    dim: int
    n: tuple
    h: float
    origin: tuple = (0.0, 0.0, 0.0)
    face_bc: tuple = (0, 0, 0, 0, 0, 0)
    face_mu: tuple = (0.0,) * 6
    g: tuple = (0.0, 0.0, 0.0)
    dt: float = 1e-5
    scheme: int = USL
    mass_tol: float = 1e-12
    face_traction: tuple = ((0.0, 0.0, 0.0),) * 6   # per face, force per unit length (area)
    damping: float = 0.0                            # alpha of a = f / m - alpha v
    face_stress: tuple = ((0.0,) * 6,) * 6          # mapped 2D mesh: uniform stress loading each face

    def c_struct(self) -> _Mesh:
        s = _Mesh()
        s.dim = self.dim
        n = list(self.n) + [1] * (3 - len(self.n))
        for k in range(3):
            s.n[k] = int(n[k])
            s.origin[k] = float(self.origin[k])
            s.g[k] = float(self.g[k])
        for f in range(6):
            s.face_bc[f] = int(self.face_bc[f])
            s.face_mu[f] = float(self.face_mu[f])
        s.h, s.dt, s.scheme, s.mass_tol = float(self.h), float(self.dt), int(self.scheme), float(self.mass_tol)
        for f in range(6):
            for k in range(3):
                s.face_traction[f][k] = float(self.face_traction[f][k])
        s.damping = float(self.damping)
        for f in range(6):
            for k in range(6):
                s.face_stress[f][k] = float(self.face_stress[f][k])
        return s

    @property
    def num_nodes(self) -> int:
        return int(lib().oracle_num_nodes(C.byref(self.c_struct())))

    def node_shape(self):
        return tuple(self.n[k] + 1 if k < self.dim else 1 for k in range(3))


@dataclass
class Material:
    model: int = LINEAR_ELASTIC
    E: float = 1e7
    nu: float = 0.3
    rho: float = 1000.0
    phi: float = 0.0
    c: float = 0.0
    psi: float = 0.0

    def c_struct(self) -> _Material:
        m = _Material()
        m.model, m.E, m.nu, m.rho, m.phi, m.c, m.psi = (int(self.model), self.E, self.nu, self.rho,
                                                      self.phi, self.c, self.psi)
        return m


@dataclass
class State:
    """Particle state, FP64, insertion order.  Vectors hold 3 components and
    stresses/strains 6 Voigt components (xx, yy, zz, xy, yz, xz) in 2D too."""
    x: np.ndarray
    v: np.ndarray
    sig: np.ndarray
    eps: np.ndarray
    m: np.ndarray
    vol: np.ndarray
    epsp: np.ndarray
    alive: np.ndarray
    coh: np.ndarray | None = None

    @classmethod
    def create(cls, pos, vel, vol, rho, sig0=None, coh=None):
        pos = np.asarray(pos, np.float64)
        n, d = pos.shape
        x = np.zeros((n, 3))
        x[:, :d] = pos
        v = np.zeros((n, 3))
        v[:, :d] = np.asarray(vel, np.float64).reshape(n, d)
        vol = np.ascontiguousarray(vol, np.float64).reshape(n).copy()
        sig = np.zeros((n, 6)) if sig0 is None else np.ascontiguousarray(sig0, np.float64).reshape(n, 6).copy()
        return cls(x=x, v=v, sig=sig, eps=np.zeros((n, 6)), m=rho * vol, vol=vol,
                   epsp=np.zeros(n), alive=np.ones(n, np.int32),
                   coh=None if coh is None else np.ascontiguousarray(coh, np.float64).reshape(n).copy())

    @property
    def n(self) -> int:
        return self.x.shape[0]

    def copy(self) -> "State":
        return State(**{k: (None if getattr(self, k) is None else getattr(self, k).copy())
                        for k in self.__dataclass_fields__})


@dataclass
class Oracle:
    """The explicit step on a Cartesian mesh, or on a mapped one when X (node
    coordinates, one row of 3 per node, x fastest) is given: then `cell`
    holds each particle's (ix, iy, iz), located at construction by the walk."""
    mesh: Mesh
    material: Material
    state: State
    _work: np.ndarray = field(default=None, repr=False)
    X: np.ndarray | None = None
    cell: np.ndarray | None = None

    def __post_init__(self):
        if self.X is not None:
            self.X = _nodes3(self.mesh, self.X)
            if self.cell is None:
                self.cell = np.zeros((self.state.n, 3), np.int32)
                c = np.zeros(3, np.int32)
                for p in range(self.state.n):    # walk on from the previous particle's cell
                    st, c, _ = locate_mapped(self.mesh, self.X, self.state.x[p], c)
                    if st != OK:
                        raise ValueError(f"particle {p} lies outside the mapped mesh")
                    self.cell[p] = c

    def step(self, nsteps: int = 1) -> int:
        L = lib()
        ms, mt = self.mesh.c_struct(), self.material.c_struct()
        if self._work is None:
            self._work = np.zeros(int(L.oracle_work_size(C.byref(ms))))
        s = self.state
        coh = _dp(s.coh) if s.coh is not None else C.cast(None, C.POINTER(C.c_double))
        if s.n == 0:
            return OK
        if self.X is not None:
            return int(L.oracle_step_mapped(C.byref(ms), _dp(self.X), C.byref(mt), s.n, _dp(s.x), _dp(s.v),
                                            _dp(s.sig), _dp(s.eps), _dp(s.m), _dp(s.vol), _dp(s.epsp), coh,
                                            _ip(s.alive), _ip(self.cell), _dp(self._work), int(nsteps)))
        return int(L.oracle_step(C.byref(ms), C.byref(mt), s.n, _dp(s.x), _dp(s.v), _dp(s.sig),
                                 _dp(s.eps), _dp(s.m), _dp(s.vol), _dp(s.epsp), coh, _ip(s.alive),
                                 _dp(self._work), int(nsteps)))

    def p2g(self):
        """Nodal mass (N,), momentum (N,3) and total force (N,3) of the state."""
        L = lib()
        ms = self.mesh.c_struct()
        nn = int(L.oracle_num_nodes(C.byref(ms)))
        nm, nP, nf = np.zeros(nn), np.zeros((nn, 3)), np.zeros((nn, 3))
        s = self.state
        L.oracle_p2g(C.byref(ms), s.n, _dp(s.x), _dp(s.v), _dp(s.sig), _dp(s.m), _dp(s.vol),
                     _ip(s.alive), _dp(nm), _dp(nP), _dp(nf))
        return nm, nP, nf

    def conservation(self):
        """mass, momentum (3,), kinetic energy, strain energy, live count."""
        s = self.state
        out = np.zeros(7)
        lib().oracle_conservation(s.n, _dp(s.v), _dp(s.sig), _dp(s.eps), _dp(s.m), _dp(s.vol),
                                  _ip(s.alive), _dp(out))
        return {"mass": out[0], "momentum": out[1:4].copy(), "ke": out[4], "se": out[5],
                "alive": int(out[6])}

    def cells(self) -> np.ndarray:
        """Integer cell (ix, iy, iz) of every particle by the oracle's locate
        rule (on a mapped mesh: the cell the walk keeps); -1 rows for
        particles outside the mesh."""
        if self.X is not None:
            return np.where(self.state.alive[:, None] == 1, self.cell, -1).astype(np.int32)
        return locate(self.mesh, self.state.x)


def locate(mesh: Mesh, x: np.ndarray):
    L = lib()
    ms = mesh.c_struct()
    x = np.ascontiguousarray(x, np.float64)
    n = x.shape[0]
    x3 = np.zeros((n, 3))
    x3[:, : x.shape[1]] = x
    cells = np.full((n, 3), -1, np.int32)
    c = np.zeros(3, np.int32)
    xi = np.zeros(3)
    for p in range(n):
        if L.oracle_locate(C.byref(ms), _dp(x3[p]), _ip(c), _dp(xi)) == OK:
            cells[p] = c
    return cells


def locate_one(mesh: Mesh, x):
    L = lib()
    x3 = np.zeros(3)
    x3[: len(x)] = x
    c = np.zeros(3, np.int32)
    xi = np.zeros(3)
    st = L.oracle_locate(C.byref(mesh.c_struct()), _dp(x3), _ip(c), _dp(xi))
    return st, c.copy(), xi.copy()


def _nodes3(mesh: Mesh, X):
    """Node coordinates as 3 per node (X may hold dim per node)."""
    X = np.asarray(X, np.float64).reshape(mesh.num_nodes, -1)
    if X.shape[1] == 3:
        return np.ascontiguousarray(X)
    out = np.zeros((mesh.num_nodes, 3))
    out[:, : X.shape[1]] = X
    return out


def natural_mapped(mesh: Mesh, X, cell, x):
    """(iterations or -1, xi (3,)) of x in a cell of a mapped mesh."""
    xi = np.zeros(3)
    x3 = np.zeros(3)
    x3[: len(x)] = x
    c = np.ascontiguousarray(cell, np.int32)
    it = lib().oracle_iso_natural(C.byref(mesh.c_struct()), _dp(_nodes3(mesh, X)), _ip(c),
                                  _dp(x3), _dp(xi))
    return int(it), xi


def locate_mapped(mesh: Mesh, X, x, start=(0, 0, 0)):
    """(status, cell (3,), xi (3,)) by the neighbourhood walk from `start`."""
    xi = np.zeros(3)
    x3 = np.zeros(3)
    x3[: len(x)] = x
    c = np.array(list(start) + [0] * (3 - len(start)), np.int32)
    st = lib().oracle_iso_locate(C.byref(mesh.c_struct()), _dp(_nodes3(mesh, X)), _dp(x3),
                                 _ip(c), _dp(xi))
    return int(st), c.copy(), xi


def face_normal(mesh: Mesh, X, face: int, ijk):
    """Outward unit normal (3,) of logical face `face` at its node ijk."""
    n = np.zeros(3)
    c = np.array(list(ijk) + [0] * (3 - len(ijk)), np.int32)
    lib().oracle_face_normal(C.byref(mesh.c_struct()), _dp(_nodes3(mesh, X)), int(face), _ip(c), _dp(n))
    return n


def basis_mapped(mesh: Mesh, X, cell, xi):
    """N (8,) and dN/dx (8, 3) at natural coordinates xi of a mapped cell."""
    N = np.zeros(8)
    G = np.zeros(24)
    x3 = np.zeros(3)
    x3[: len(xi)] = xi
    lib().oracle_iso_basis(C.byref(mesh.c_struct()), _dp(_nodes3(mesh, X)),
                           _ip(np.ascontiguousarray(cell, np.int32)), _dp(x3), _dp(N), _dp(G))
    return N, G.reshape(8, 3)


def shape(dim: int, xi):
    """N (8,) and dN/dxi (8,3) at natural coordinates xi."""
    x = np.zeros(3)
    x[: len(xi)] = xi
    N = np.zeros(8)
    dN = np.zeros(24)
    lib().oracle_shape(dim, _dp(x), _dp(N), _dp(dN))
    return N, dN.reshape(8, 3)


def eig_sym3(s6):
    s = np.ascontiguousarray(s6, np.float64)
    lam = np.zeros(3)
    V = np.zeros(9)
    lib().oracle_eig_sym3(_dp(s), _dp(lam), _dp(V))
    return lam, V.reshape(3, 3)


def mc_return(E, nu, phi, psi, c, sig_tr):
    """Mohr-Coulomb return of one trial stress: (sigma (6,), branch, depsp)."""
    s = np.ascontiguousarray(sig_tr, np.float64)
    out = np.zeros(6)
    d = np.zeros(1)
    br = lib().oracle_mc_return(E, nu, phi, psi, c, _dp(s), _dp(out), _dp(d))
    return out, int(br), float(d[0])


def stress_update(material: Material, coh: float, sig, de):
    s = np.array(sig, np.float64)
    d = np.ascontiguousarray(de, np.float64)
    e = np.zeros(1)
    lib().oracle_stress_update(C.byref(material.c_struct()), coh, _dp(s), _dp(d), _dp(e))
    return s, float(e[0])


def constrain_node(mesh: Mesh, ijk, v, a, vn):
    v = np.array(v, np.float64)
    a = np.array(a, np.float64)
    vn = np.array(vn, np.float64)
    c = np.array(ijk, np.int32)
    lib().oracle_constrain_node(C.byref(mesh.c_struct()), _ip(c), _dp(v), _dp(a), _dp(vn))
    return v, a, vn


def from_workload(wl, scheme=None) -> Oracle:
    """Oracle on a workload from paper_1909_13380_gb300.workloads (inputs only)."""
    mesh = Mesh(dim=wl.dim, n=wl.ncells, h=wl.h, origin=wl.origin, face_bc=wl.face_bc, face_mu=wl.face_mu,
                g=wl.gravity, dt=wl.dt, scheme=wl.scheme if scheme is None else scheme,
                face_traction=wl.face_traction, damping=wl.damping,
                face_stress=getattr(wl, "face_stress", ((0.0,) * 6,) * 6))
    st = State.create(wl.pos, wl.vel, wl.vol, wl.material["rho"], coh=wl.coh)
    return Oracle(mesh, Material(**wl.material), st, X=getattr(wl, "node_xyz", None))
