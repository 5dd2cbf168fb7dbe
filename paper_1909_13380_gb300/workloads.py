"""Seeded synthetic inputs shaped like the workloads of the explicit MPM path.

This module only lays out geometry and draws random numbers: where particles
sit, their initial velocity and volume, the mesh and boundary description and
the material constants.  It holds none of the method's arithmetic, and both
the CUDA library and the FP64 oracle take their inputs from it unchanged.

Every generator is deterministic: randomness comes from numpy's PCG64 seeded
with ``1909133800 + k`` for workload ``k``.

Face numbering (-x, +x, -y, +y, -z, +z) and boundary codes follow the C-ABI:
FREE 0, ROLLER 1, FIXED 2, FRICTION 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FREE, ROLLER, FIXED, FRICTION = 0, 1, 2, 3
USF, USL = 0, 1
FP64_PLAIN, FP32_MIXED = 0, 1
LINEAR_ELASTIC, MOHR_COULOMB, PLANE_STRESS_ELASTIC = 0, 1, 2
SEED_BASE = 1909133800


@dataclass
class Workload:
    name: str
    dim: int
    ncells: tuple
    h: float
    origin: tuple
    face_bc: tuple
    face_mu: tuple
    gravity: tuple
    dt: float
    scheme: int
    precision: int
    material: dict            # model, E, nu, rho, phi (rad), c, psi (rad)
    pos: np.ndarray           # (n, dim) float64
    vel: np.ndarray           # (n, dim) float64
    vol: np.ndarray           # (n,) float64
    coh: np.ndarray | None = None   # (n,) float64 per-particle cohesion, or None
    steps: int = 1
    meta: dict = field(default_factory=dict)
    face_traction: tuple = ((0.0, 0.0, 0.0),) * 6   # per face: force per unit length (2D) or area (3D)
    damping: float = 0.0                            # alpha of the nodal damping a = f / m - alpha v
    node_xyz: np.ndarray | None = None              # mapped mesh: (nodes, dim) node coordinates, x fastest
    face_stress: tuple = ((0.0,) * 6,) * 6          # mapped 2D mesh: uniform stress (Voigt) loading each face

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def num_nodes(self) -> int:
        k = 1
        for d in range(self.dim):
            k *= self.ncells[d] + 1
        return k


def gauss_fill(cells: np.ndarray, h: float, origin, dim: int) -> np.ndarray:
    """Two particles per axis in every listed cell, at the cell centre
    +- h / (2 sqrt 3) (the 2-point Gauss positions).  Cells are visited in the
    given order and the 2^dim points of a cell x fastest."""
    cells = np.asarray(cells, np.int64).reshape(-1, dim)
    g = 0.5 / math.sqrt(3.0)
    offs = np.array([[(g if (a >> k) & 1 else -g) for k in range(dim)] for a in range(1 << dim)])
    centres = (cells.astype(np.float64) + 0.5) * h + np.asarray(origin[:dim], np.float64)
    pos = centres[:, None, :] + offs[None, :, :] * h
    return pos.reshape(-1, dim)


def box_cells(lo, hi) -> np.ndarray:
    """All integer cells lo <= c < hi (per axis), x fastest."""
    axes = [np.arange(l, u) for l, u in zip(lo, hi)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)


def _mc(phi_deg=30.0, c=0.0, psi_deg=0.0, E=10e6, nu=0.3, rho=1800.0):
    return dict(model=MOHR_COULOMB, E=E, nu=nu, rho=rho, phi=math.radians(phi_deg), c=c,
                psi=math.radians(psi_deg))


def elastic_bar(precision: int = FP64_PLAIN, scheme: int = USF, steps: int = 2000) -> Workload:
    """2D plane-strain bar, 64 x 4 quads of 0.1 m filled with 2 x 2 Gauss
    particles (1024), E = 100 MPa, nu = 0, rho = 1000, left edge fixed, no
    gravity, initial axial velocity v0 sin(pi x / 2L), v0 = 0.1 m/s."""
    nx, ny, h = 64, 4, 0.1
    L = nx * h
    pos = gauss_fill(box_cells((0, 0), (nx, ny)), h, (0.0, 0.0), 2)
    vel = np.zeros_like(pos)
    vel[:, 0] = 0.1 * np.sin(np.pi * pos[:, 0] / (2.0 * L))
    vol = np.full(pos.shape[0], h * h / 4.0)
    return Workload(
        name="elastic_bar_2d_64x4", dim=2, ncells=(nx, ny, 1), h=h, origin=(0.0, 0.0, 0.0),
        face_bc=(FIXED, FREE, FREE, FREE, FREE, FREE), face_mu=(0.0,) * 6, gravity=(0.0, 0.0, 0.0),
        dt=1e-5, scheme=scheme, precision=precision,
        material=dict(model=LINEAR_ELASTIC, E=100e6, nu=0.0, rho=1000.0, phi=0.0, c=0.0, psi=0.0),
        pos=pos, vel=vel, vol=vol, steps=steps, meta=dict(L=L, v0=0.1))


def column3d(ncells=(200, 40, 100), col_cells=(40, 40, 40), h=0.005, precision=FP32_MIXED,
             scheme=USL, steps=5000, name=None) -> Workload:
    """3D dry granular column collapse on 8-node hexahedra: a column of
    col_cells at the (x=0, y=0, z=0) corner filled with 8 Gauss particles per
    cell; Mohr-Coulomb phi 30 deg, c 0, psi 0, E 10 MPa, nu 0.3, rho 1800;
    gravity 9.81 along -z; rollers at x = 0 and both y faces, Coulomb base
    mu = 0.4, free top and +x.  The default sizes are the 200 x 40 x 100 mesh
    of 5 mm cells with a 0.2 m cube column (512,000 particles)."""
    pos = gauss_fill(box_cells((0, 0, 0), col_cells), h, (0.0, 0.0, 0.0), 3)
    vel = np.zeros_like(pos)
    vol = np.full(pos.shape[0], h ** 3 / 8.0)
    nm = name or f"granular_column_3d_{ncells[0]}x{ncells[1]}x{ncells[2]}_col{col_cells[0]}x{col_cells[1]}x{col_cells[2]}"
    return Workload(
        name=nm, dim=3, ncells=tuple(ncells), h=h, origin=(0.0, 0.0, 0.0),
        face_bc=(ROLLER, FREE, ROLLER, ROLLER, FRICTION, FREE), face_mu=(0, 0, 0, 0, 0.4, 0),
        gravity=(0.0, 0.0, -9.81), dt=1e-5, scheme=scheme, precision=precision, material=_mc(),
        pos=pos, vel=vel, vol=vol, steps=steps)


def column2d(width_cells: int, height_cells: int, h=0.0025, precision=FP32_MIXED, scheme=USL,
             mesh_cells=None, steps=5000, name=None) -> Workload:
    """2D plane-strain granular column (4 Gauss particles per quad) against
    the left wall; rollers at both x faces, Coulomb base mu = 0.4; the same
    Mohr-Coulomb set as the 3D column."""
    W, H = int(width_cells), int(height_cells)
    if mesh_cells is None:
        mesh_cells = (3 * W + 2, H + 4)
    pos = gauss_fill(box_cells((0, 0), (W, H)), h, (0.0, 0.0), 2)
    vel = np.zeros_like(pos)
    vol = np.full(pos.shape[0], h * h / 4.0)
    return Workload(
        name=name or f"granular_column_2d_{W}x{H}", dim=2, ncells=(mesh_cells[0], mesh_cells[1], 1), h=h,
        origin=(0.0, 0.0, 0.0), face_bc=(ROLLER, ROLLER, FRICTION, FREE, FREE, FREE),
        face_mu=(0, 0, 0.4, 0, 0, 0), gravity=(0.0, -9.81, 0.0), dt=1e-5, scheme=scheme,
        precision=precision, material=_mc(), pos=pos, vel=vel, vol=vol, steps=steps)


def columns2d_batch(count=256, seed=SEED_BASE + 3, h=0.0025, steps=5000):
    """A set of independent 2D granular columns: particle count log-uniform
    in [5e3, 6e4], aspect ratio uniform in [0.5, 4]; width W = round(sqrt(n /
    (4a))) cells, height H = round(a W); mesh (2 + 3a) W by H + 4 cells."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = float(np.exp(rng.uniform(np.log(5e3), np.log(6e4))))
        a = float(rng.uniform(0.5, 4.0))
        W = max(1, int(round(math.sqrt(n / (4.0 * a)))))
        H = max(1, int(round(a * W)))
        mesh = (int(round((2.0 + 3.0 * a) * W)), H + 4)
        out.append(column2d(W, H, h=h, mesh_cells=mesh, steps=steps, name=f"column2d_{i}_{W}x{H}"))
    return out


def slope3d(ncells=(800, 200, 200), h=0.05, crest=8.0, plateau=8.5, seed=SEED_BASE + 5,
            precision=FP32_MIXED, steps=2000) -> Workload:
    """3D slope on hexahedra: the x-z section is a plateau of height `crest`
    from x = 0 to `plateau`, then a 45-degree face down to z = 0, extruded
    over the whole y width.  A cell is filled when its centre lies inside the
    section; 8 Gauss particles per filled cell.  Cohesion: one lognormal draw
    (mean 10 kPa, CoV 0.3) per filled cell in cell order, shared by its
    particles.  phi 30 deg, psi 0, E 50 MPa, nu 0.3, rho 2000; fixed base,
    rollers on the four sides, free top."""
    nx, ny, nz = ncells
    ix = np.arange(nx)
    iz = np.arange(nz)
    xc = (ix + 0.5) * h
    zc = (iz + 0.5) * h
    top = np.where(xc <= plateau, crest, crest - (xc - plateau))          # surface height at xc
    inside = zc[:, None] < top[None, :]                                     # (nz, nx)
    zz, xx = np.nonzero(inside)                                             # z-major, x fastest
    nxz = xx.shape[0]
    cells = np.empty((nxz * ny, 3), np.int64)
    # cell order x fastest, then y, then z (lexicographic cell id order)
    order = []
    for k in np.unique(zz):
        xs = xx[zz == k]
        for j in range(ny):
            order.append(np.stack([xs, np.full_like(xs, j), np.full_like(xs, k)], axis=1))
    cells = np.concatenate(order, axis=0)
    rng = np.random.Generator(np.random.PCG64(seed))
    sig_ln = math.sqrt(math.log(1.0 + 0.3 ** 2))
    mu_ln = math.log(10e3) - 0.5 * sig_ln ** 2
    coh_cell = rng.lognormal(mu_ln, sig_ln, size=cells.shape[0])
    pos = gauss_fill(cells, h, (0.0, 0.0, 0.0), 3)
    coh = np.repeat(coh_cell, 8)
    vel = np.zeros_like(pos)
    vol = np.full(pos.shape[0], h ** 3 / 8.0)
    return Workload(
        name=f"slope_3d_{nx}x{ny}x{nz}", dim=3, ncells=(nx, ny, nz), h=h, origin=(0.0, 0.0, 0.0),
        face_bc=(ROLLER, ROLLER, ROLLER, ROLLER, FIXED, FREE), face_mu=(0.0,) * 6,
        gravity=(0.0, 0.0, -9.81), dt=1e-5, scheme=USL, precision=precision,
        material=_mc(E=50e6, rho=2000.0, c=10e3), pos=pos, vel=vel, vol=vol, coh=coh, steps=steps,
        meta=dict(crest=crest, plateau=plateau, filled_cells=int(cells.shape[0])))


def slope2d(ncells, h=0.05, crest=8.0, plateau=8.5, seed=SEED_BASE + 6, precision=FP32_MIXED,
            steps=2000, name=None) -> Workload:
    """2D plane-strain slope on quads, the x-y section of `slope3d` (y up):
    plateau of height `crest` up to x = `plateau`, then a 45-degree face;
    4 Gauss particles per filled cell; lognormal cohesion per filled cell
    (mean 10 kPa, CoV 0.3); fixed base, rollers on both sides."""
    nx, ny = ncells[0], ncells[1]
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h
    top = np.where(xc <= plateau, crest, crest - (xc - plateau))
    inside = yc[:, None] < top[None, :]                                     # (ny, nx)
    yy, xx = np.nonzero(inside)                                             # y-major, x fastest
    cells = np.stack([xx, yy], axis=1)
    rng = np.random.Generator(np.random.PCG64(seed))
    sig_ln = math.sqrt(math.log(1.0 + 0.3 ** 2))
    mu_ln = math.log(10e3) - 0.5 * sig_ln ** 2
    coh = np.repeat(rng.lognormal(mu_ln, sig_ln, size=cells.shape[0]), 4)
    pos = gauss_fill(cells, h, (0.0, 0.0), 2)
    vel = np.zeros_like(pos)
    vol = np.full(pos.shape[0], h * h / 4.0)
    return Workload(
        name=name or f"slope_2d_{nx}x{ny}", dim=2, ncells=(nx, ny, 1), h=h, origin=(0.0, 0.0, 0.0),
        face_bc=(ROLLER, ROLLER, FIXED, FREE, FREE, FREE), face_mu=(0.0,) * 6,
        gravity=(0.0, -9.81, 0.0), dt=1e-5, scheme=USL, precision=precision,
        material=_mc(E=50e6, rho=2000.0, c=10e3), pos=pos, vel=vel, vol=vol, coh=coh, steps=steps,
        meta=dict(crest=crest, plateau=plateau, filled_cells=int(cells.shape[0])))


REQUEST_KINDS = ("column2d", "column3d", "slope2d", "slope3d")


def request_workload(kind: str, n_target: float, seed: int, steps: int, precision=FP32_MIXED) -> Workload:
    """One serving request of about `n_target` particles.
      column2d  aspect a ~ U[0.5, 4]; W = sqrt(n / 4a), H = a W cells of 2.5 mm
      column3d  aspect a ~ U[0.5, 4]; W x W x aW cells of 5 mm, mesh as the
                200 x 40 x 100 column ((2 + 3a) W long, W wide, H + 4 high)
      slope2d   plateau and face of height Hc, Hc = sqrt(n / 6) cells of 5 cm
      slope3d   the same section extruded over Hc / 2 cells."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = float(n_target)
    if kind == "column2d":
        a = float(rng.uniform(0.5, 4.0))
        W = max(1, int(round(math.sqrt(n / (4.0 * a)))))
        H = max(1, int(round(a * W)))
        return column2d(W, H, mesh_cells=(int(round((2.0 + 3.0 * a) * W)), H + 4), precision=precision,
                        steps=steps, name=f"column2d_{W}x{H}")
    if kind == "column3d":
        a = float(rng.uniform(0.5, 4.0))
        W = max(1, int(round((n / (8.0 * a)) ** (1.0 / 3.0))))
        H = max(1, int(round(a * W)))
        return column3d(ncells=(int(round((2.0 + 3.0 * a) * W)), W, H + 4), col_cells=(W, W, H),
                        precision=precision, steps=steps, name=f"column3d_{W}x{W}x{H}")
    hs = 0.05
    if kind == "slope2d":
        Hc = max(2, int(round(math.sqrt(n / 6.0))))
        return slope2d((2 * Hc + Hc // 2, Hc + 4), h=hs, crest=Hc * hs, plateau=Hc * hs,
                       seed=int(rng.integers(1 << 31)), precision=precision, steps=steps,
                       name=f"slope2d_H{Hc}")
    if kind == "slope3d":
        Hc = max(2, int(round((n / 6.0) ** (1.0 / 3.0))))
        wl = slope3d(ncells=(2 * Hc + Hc // 2, max(1, Hc // 2), Hc + 4), h=hs, crest=Hc * hs, plateau=Hc * hs,
                     seed=int(rng.integers(1 << 31)), precision=precision, steps=steps)
        wl.name = f"slope3d_H{Hc}"
        return wl
    raise ValueError(kind)


@dataclass
class Request:
    rid: int
    arrival: float      # seconds after the start of the session
    kind: str
    n_target: int
    steps: int
    seed: int

    def workload(self, precision=FP32_MIXED) -> Workload:
        return request_workload(self.kind, self.n_target, self.seed, self.steps, precision)


def serving_requests(count=32, rate=20.0, n_range=(1e4, 4e6), steps_range=(1000, 20000), step_scale=1.0 / 50,
                     seed=SEED_BASE + 4, kinds=REQUEST_KINDS):
    """A Poisson stream of mixed requests: exponential inter-arrival times of
    mean 1 / rate, kind uniform over `kinds`, particle count and step count
    log-uniform over their ranges; the step count is then multiplied by
    `step_scale` (at least 1), which keeps a bounded session's offered load
    below the GPU's capacity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = kinds[int(rng.integers(len(kinds)))]
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        st = math.exp(rng.uniform(math.log(steps_range[0]), math.log(steps_range[1])))
        steps = max(1, int(round(st * step_scale)))
        out.append(Request(i, t, kind, n, steps, int(rng.integers(1 << 31))))
    return out


def random_particles(mesh_cells, h, n, seed, dim=3, margin=1, vel_scale=0.1, sig_scale=1e3):
    """Uniform random particle positions inside the mesh (away from the
    boundary by `margin` cells), random velocity and random symmetric stress:
    inputs for brute-force and parity checks of a single transfer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.array([margin * h] * dim)
    hi = np.array([(mesh_cells[k] - margin) * h for k in range(dim)])
    pos = lo + (hi - lo) * rng.random((n, dim))
    vel = vel_scale * rng.standard_normal((n, dim))
    sig = np.zeros((n, 6))
    if dim == 3:
        sig[:] = sig_scale * rng.standard_normal((n, 6))
    else:
        sig[:, :4] = sig_scale * rng.standard_normal((n, 4))
    vol = (h ** dim / 4.0) * (0.5 + rng.random(n))
    return pos, vel, sig, vol


def plate_with_hole(h=0.0625, per_axis=4, E=1e6, nu=0.3, rho=1000.0, sigma0=100.0, radius=0.5,
                    precision=FP64_PLAIN, scheme=USF, dt=None, damping=None, steps=4000) -> Workload:
    """The validation problem of the paper's benchmark: a plane-stress strip
    8 m long and 5 m wide with a centred hole of radius 0.5 m under uniform
    tension sigma0 at its ends, modelled by its quarter x in [0, 4],
    y in [0, 2.5] (the hole's centre at the origin): rollers on x = 0 and
    y = 0 (symmetry), the traction (sigma0, 0) on the +x face, cells of
    0.0625 m filled with per_axis^2 = 16 particles each at the centres of a
    regular sub-grid, the particles inside the hole left out (40,156
    particles).  The elastic constants do not change the static stress
    field; dt is a fifth of the time a plane-stress wave takes to cross a
    cell, and the viscous damping alpha (a = f / m - alpha v) twice the
    lowest frequency of a fixed-free bar of the strip's half length."""
    nx, ny = int(round(4.0 / h)), int(round(2.5 / h))
    cells = box_cells((0, 0), (nx, ny)).astype(np.float64)
    sub = (np.arange(per_axis) + 0.5) / per_axis
    sx, sy = np.meshgrid(sub, sub, indexing="xy")
    offs = np.stack([sx.ravel(), sy.ravel()], axis=1)
    pos = ((cells[:, None, :] + offs[None, :, :]) * h).reshape(-1, 2)
    pos = pos[pos[:, 0] ** 2 + pos[:, 1] ** 2 >= radius ** 2]
    vol = np.full(pos.shape[0], (h / per_axis) ** 2)
    c = math.sqrt(E / (rho * (1.0 - nu * nu)))
    if dt is None:
        dt = 0.2 * h / c
    if damping is None:
        damping = 2.0 * math.pi * c / (2.0 * 4.0)
    trac = [(0.0, 0.0, 0.0)] * 6
    trac[1] = (sigma0, 0.0, 0.0)
    return Workload(
        name=f"plate_with_hole_quarter_{nx}x{ny}", dim=2, ncells=(nx, ny, 1), h=h, origin=(0.0, 0.0, 0.0),
        face_bc=(ROLLER, FREE, ROLLER, FREE, FREE, FREE), face_mu=(0.0,) * 6, gravity=(0.0, 0.0, 0.0), dt=dt,
        scheme=scheme, precision=precision,
        material=dict(model=PLANE_STRESS_ELASTIC, E=E, nu=nu, rho=rho, phi=0.0, c=0.0, psi=0.0),
        pos=pos, vel=np.zeros_like(pos), vol=vol, steps=steps, face_traction=tuple(trac), damping=damping,
        meta=dict(sigma0=sigma0, radius=radius))


# ---------------------------------------------------------------------------
# Mapped (isoparametric) meshes: the logical grid of cells is the Cartesian
# one, the nodes are moved (ISOPARAMETRIC MESH: non-prismatic boundaries).
# ---------------------------------------------------------------------------
def cartesian_node_xyz(ncells, h, origin=(0.0, 0.0, 0.0), dim=3) -> np.ndarray:
    """Node coordinates of the Cartesian grid, one row per node, x fastest."""
    axes = [origin[k] + h * np.arange(ncells[k] + 1) for k in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)


def rotation(dim: int, angles) -> np.ndarray:
    """Rotation matrix: angle (2D), or rotations about x, then y, then z (3D)."""
    if dim == 2:
        c, s = math.cos(angles), math.sin(angles)
        return np.array([[c, -s], [s, c]])
    ax, ay, az = angles
    Rx = np.array([[1, 0, 0], [0, math.cos(ax), -math.sin(ax)], [0, math.sin(ax), math.cos(ax)]])
    Ry = np.array([[math.cos(ay), 0, math.sin(ay)], [0, 1, 0], [-math.sin(ay), 0, math.cos(ay)]])
    Rz = np.array([[math.cos(az), -math.sin(az), 0], [math.sin(az), math.cos(az), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def rotated(wl: Workload, R: np.ndarray, name=None) -> Workload:
    """The same problem turned rigidly about the origin: a mapped mesh whose
    nodes, particles, velocities and gravity are the Cartesian ones times R.
    Boundary faces must be free or fixed (a turned roller acts along the
    logical face's axis)."""
    d = wl.dim
    X = cartesian_node_xyz(wl.ncells, wl.h, wl.origin, d) @ R.T
    g = np.zeros(3)
    g[:d] = np.asarray(wl.gravity[:d]) @ R.T
    return Workload(**{**wl.__dict__, "name": name or wl.name + "_rotated", "pos": wl.pos @ R.T,
                       "vel": wl.vel @ R.T, "gravity": tuple(g), "node_xyz": X})


def terrain(points: np.ndarray, dim: int, amp: float, wavelength: float, height: float) -> np.ndarray:
    """The terrain-following map of a box of the given height: the vertical
    coordinate v -> v + b(x) (1 - v / height), b(x) = amp sin(2 pi x / wavelength),
    so the base follows the bumps b and the top stays flat."""
    p = np.array(points, np.float64)
    up = dim - 1
    b = amp * np.sin(2.0 * math.pi * p[:, 0] / wavelength)
    p[:, up] = p[:, up] + b * (1.0 - p[:, up] / height)
    return p


def terrain_column(dim=2, ncells=None, col_cells=None, h=0.005, amp=None, wavelength=None,
                   precision=FP64_PLAIN, scheme=USL, steps=2000, name=None) -> Workload:
    """A granular column collapsing on bumpy ground: the mesh follows the
    terrain (mapped cells, the base a sine of amplitude amp), the column's
    particles are the Cartesian 2-point Gauss positions moved by the same
    map.  Mohr-Coulomb as the 3D column; a Coulomb base (mu 0.4) along the
    bumpy ground's normals, a roller on x = 0 (a vertical plane under the
    map), the other faces free."""
    if ncells is None:
        ncells = (60, 24) if dim == 2 else (40, 8, 24)
    if col_cells is None:
        col_cells = (12, 12) if dim == 2 else (12, 8, 12)
    nodes = ncells[: dim]
    height = nodes[dim - 1] * h
    amp = 2.5 * h if amp is None else amp
    wavelength = 16.0 * h if wavelength is None else wavelength
    cells = box_cells((0,) * dim, col_cells)
    flat = gauss_fill(cells, h, (0.0, 0.0, 0.0), dim)
    pos = terrain(flat, dim, amp, wavelength, height)
    # the map stretches the vertical by 1 - b(x) / height (its Jacobian
    # determinant): each particle keeps that share of its Gauss volume
    stretch = 1.0 - amp * np.sin(2.0 * math.pi * flat[:, 0] / wavelength) / height
    X = terrain(cartesian_node_xyz(ncells, h, (0.0, 0.0, 0.0), dim), dim, amp, wavelength, height)
    bc = [FREE] * 6
    bc[0] = ROLLER
    bc[2 * (dim - 1)] = FRICTION
    mu = [0.0] * 6
    mu[2 * (dim - 1)] = 0.4
    g = [0.0, 0.0, 0.0]
    g[dim - 1] = -9.81
    nm = name or f"terrain_column_{dim}d_" + "x".join(str(c) for c in ncells[:dim])
    return Workload(
        name=nm, dim=dim, ncells=tuple(ncells[:dim]) + (1,) * (3 - dim), h=h, origin=(0.0, 0.0, 0.0),
        face_bc=tuple(bc), face_mu=tuple(mu), gravity=tuple(g), dt=1e-5, scheme=scheme, precision=precision,
        material=_mc(), pos=pos, vel=np.zeros_like(pos), vol=stretch * h ** dim / (1 << dim),
        steps=steps, node_xyz=X, meta=dict(amp=amp, wavelength=wavelength))


def warp(points: np.ndarray, dim: int, h: float, amp: float = 0.2, wavelength: float = 7.0) -> np.ndarray:
    """A smooth warp of space: coordinate k moves by amp h sin(2 pi x_j /
    (wavelength h) + 0.7 k), j the next axis; its Jacobian stays within
    2 pi amp / wavelength of the identity, so warped cells keep their
    orientation."""
    p = np.array(points, np.float64)
    out = p.copy()
    w = 2.0 * math.pi / (wavelength * h)
    for k in range(dim):
        out[:, k] += amp * h * np.sin(w * p[:, (k + 1) % dim] + 0.7 * k)
    return out


def warped_box(ncells=(12, 10, 8), h=0.1, n=3000, seed=SEED_BASE + 51, dim=3, scheme=USL, steps=100,
               drift=(1.0, 0.6, -0.4), name=None) -> Workload:
    """Elastic particles scattered in a box whose nodes are moved by warp():
    a mapped mesh of curved-sided cells.  The particles (uniform random,
    2 cells clear of the boundary, where the mesh's piecewise-linear faces
    depart from the warp) are moved by the same warp; they drift at `drift`
    m/s (about a cell per 100 steps) plus a small random velocity, with a
    random initial stress (meta["stress0"]); a soft solid (E = 10 kPa: the
    elastic wave crosses a cell in several steps), free faces, no gravity."""
    ncells = tuple(ncells[:dim])
    pos, vel, sig, vol = random_particles(ncells, h, n, seed, dim=dim, margin=2, vel_scale=0.05, sig_scale=10.0)
    pos = warp(pos, dim, h)
    vel = vel + np.asarray(drift[:dim])
    X = warp(cartesian_node_xyz(ncells + (1,) * (3 - dim), h, (0.0, 0.0, 0.0), dim), dim, h)
    nm = name or f"warped_box_{dim}d_" + "x".join(str(c) for c in ncells)
    return Workload(
        name=nm, dim=dim, ncells=ncells + (1,) * (3 - dim), h=h, origin=(0.0, 0.0, 0.0), face_bc=(FREE,) * 6,
        face_mu=(0.0,) * 6, gravity=(0.0, 0.0, 0.0), dt=1e-3, scheme=scheme, precision=FP64_PLAIN,
        material=dict(model=LINEAR_ELASTIC, E=1e4, nu=0.3, rho=1000.0, phi=0.0, c=0.0, psi=0.0),
        pos=pos, vel=vel, vol=vol, steps=steps, node_xyz=X, meta=dict(stress0=sig))


def ogrid_map(i, j, nr, nt, radius=0.5, length=4.0, width=2.5, grading=3.0):
    """The quarter plate with a hole as one logical grid (an O-grid): logical
    (i, j) in [0, nr] x [0, nt] (reals) to the plane.  j runs around the
    hole's circle at uniform angle (0 to 90 degrees) and along the outer
    boundary -- up the loaded end x = length (y from 0 to width), then along
    the free edge y = width back to x = 0 -- with nodes spread in proportion to
    the two lengths; i runs along the segment joining the two, graded towards
    the hole: s = (exp(grading i / nr) - 1) / (exp(grading) - 1)."""
    i = np.asarray(i, np.float64)
    j = np.asarray(j, np.float64)
    n1 = max(1, int(round(nt * width / (width + length))))
    up = j <= n1
    ox = np.where(up, length, length - length * (j - n1) / (nt - n1))
    oy = np.where(up, width * j / n1, width)
    th = 0.5 * math.pi * j / nt
    ix, iy = radius * np.cos(th), radius * np.sin(th)
    s = np.expm1(grading * i / nr) / math.expm1(grading)
    return np.stack([ix + s * (ox - ix), iy + s * (oy - iy)], axis=-1)


def plate_with_hole_ogrid(nr=20, nt=32, per_axis=2, grading=3.5, E=1e6, nu=0.3, rho=1000.0, sigma0=100.0, radius=0.5,
                          precision=FP64_PLAIN, scheme=USF, steps=None, damping=None, cfl=0.4) -> Workload:
    """The plate of plate_with_hole on a mapped mesh that fits the hole: the
    O-grid of ogrid_map (nr cells along the rays, nt around), the logical
    faces -x the hole (free), -y the symmetry line y = 0 and +y the symmetry
    line x = 0 (rollers along their normals), +x the loaded end and the free
    edge, loaded by the far-field stress sigma0 e_x e_x (traction sigma0 on
    the end, none on the edge).  per_axis^2 particles per cell at the regular
    sub-grid of its logical square, placed and weighted (volume = the map's
    Jacobian times the logical area) by the smooth map.  Plane stress; dt the
    fraction cfl of the wave's crossing time of the smallest cell edge,
    damping as plate_with_hole's, run for the same physical time; h (a
    length unit only, on a mapped mesh) the longest cell edge."""
    I, J = np.meshgrid(np.arange(nr + 1), np.arange(nt + 1), indexing="xy")
    X = ogrid_map(I.ravel(), J.ravel(), nr, nt, radius, grading=grading).reshape(-1, 2)
    sub = (np.arange(per_axis) + 0.5) / per_axis
    ci, cj = np.meshgrid(np.arange(nr), np.arange(nt), indexing="xy")
    li = (ci.ravel()[:, None, None] + sub[None, None, :]).repeat(per_axis, axis=1)
    lj = (cj.ravel()[:, None, None] + sub[None, :, None]).repeat(per_axis, axis=2)
    li, lj = li.ravel(), lj.ravel()
    om = lambda a, b: ogrid_map(a, b, nr, nt, radius, grading=grading)  # noqa: E731
    pos = om(li, lj)
    eps = 1e-6
    dxi = (om(li + eps, lj) - om(li - eps, lj)) / (2 * eps)
    dxj = (om(li, lj + eps) - om(li, lj - eps)) / (2 * eps)
    vol = np.abs(dxi[:, 0] * dxj[:, 1] - dxi[:, 1] * dxj[:, 0]) / per_axis ** 2
    Xg = X.reshape(nt + 1, nr + 1, 2)
    edges = np.concatenate([np.linalg.norm(np.diff(Xg, axis=0), axis=-1).ravel(),
                            np.linalg.norm(np.diff(Xg, axis=1), axis=-1).ravel()])
    c = math.sqrt(E / (rho * (1.0 - nu * nu)))
    dt = cfl * edges.min() / c
    if damping is None:
        damping = 2.0 * math.pi * c / (2.0 * 4.0)
    if steps is None:   # plate_with_hole's 4000 steps of 0.2 h / c, h = 0.0625
        steps = int(math.ceil(4000 * 0.2 * 0.0625 / c / dt))
    fs = [(0.0,) * 6] * 6
    fs[1] = (sigma0, 0.0, 0.0, 0.0, 0.0, 0.0)
    return Workload(
        name=f"plate_with_hole_ogrid_{nr}x{nt}", dim=2, ncells=(nr, nt, 1), h=edges.max(), origin=(0.0, 0.0, 0.0),
        face_bc=(FREE, FREE, ROLLER, ROLLER, FREE, FREE), face_mu=(0.0,) * 6, gravity=(0.0, 0.0, 0.0), dt=dt,
        scheme=scheme, precision=precision,
        material=dict(model=PLANE_STRESS_ELASTIC, E=E, nu=nu, rho=rho, phi=0.0, c=0.0, psi=0.0),
        pos=pos, vel=np.zeros_like(pos), vol=vol, steps=steps, damping=damping, node_xyz=X, face_stress=tuple(fs),
        meta=dict(sigma0=sigma0, radius=radius))
