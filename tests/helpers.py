"""Test helpers: oracle set-up from a workload, GPU state -> oracle state, and
the relative-L2 comparisons used by the parity tests.

Tolerances (relative L2 over all particles and components):
  FP64 GPU vs FP64 oracle: 1e-9 after the run (only summation order differs);
  FP32 mixed vs FP64 oracle: 1e-5 for one step from an identical state, 1e-3
  after a full run.
Positions and volumes are compared as increments over the compared window
(their absolute values would hide the error), velocities and stresses as they
are.
"""
import math

import numpy as np

import oracle
from paper_1909_13380_gb300 import workloads as W

TOL_STEP_FP32 = 1e-5
TOL_RUN_FP32 = 1e-3
TOL_RUN_FP64 = 1e-9


def oracle_from_workload(wl, scheme=None):
    return oracle.from_workload(wl, scheme)


def oracle_from_gpu(wl, snap, scheme=None):
    """Oracle whose particle state is a GPU snapshot (insertion order)."""
    o = oracle_from_workload(wl, scheme)
    s = o.state
    d = wl.dim
    s.x[:, :d] = snap["pos"]
    s.v[:, :d] = snap["vel"]
    s.sig[:] = snap["stress"]
    s.eps[:] = snap["strain"]
    s.vol[:] = snap["vol"]
    s.epsp[:] = snap["epsp"]
    s.alive[:] = (snap["cell"] >= 0).astype(np.int32)
    return o


def oracle_snapshot(o, dim):
    s = o.state
    cells = o.cells()
    nc = o.mesh.n
    lin = np.where(cells[:, 0] >= 0, cells[:, 0] + nc[0] * (cells[:, 1] + nc[1] * cells[:, 2]), -1)
    return {"pos": s.x[:, :dim].copy(), "vel": s.v[:, :dim].copy(), "stress": s.sig.copy(),
            "strain": s.eps.copy(), "vol": s.vol.copy(), "epsp": s.epsp.copy(), "cell": lin}


def rel_l2(a, b, floor=0.0):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = max(np.linalg.norm(b), floor)
    if den == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / den)


STATE_KEYS = ("pos", "vel", "stress", "vol")     # per-step check: the state itself
RUN_KEYS = ("disp", "vel", "stress", "dvol")      # after a run: increments too


def compare(gpu, ref, start, dim, h=None):
    """Relative-L2 errors of a GPU snapshot against the oracle's.

    pos/vol: the state (positions measured from the mesh origin);
    disp/dvol: increments since `start`, the common initial snapshot -- a
    single FP32 step moves a particle by ~1e-5 cells, close to the 3e-8-cell
    resolution of its FP32 offset, so increments are only meaningful over a
    run; off_cells: largest position difference in cell units."""
    live = (gpu["cell"] >= 0) & (ref["cell"] >= 0)
    out = {
        "pos": rel_l2(gpu["pos"][live], ref["pos"][live]),
        "disp": rel_l2((gpu["pos"] - start["pos"])[live], (ref["pos"] - start["pos"])[live]),
        "vel": rel_l2(gpu["vel"][live], ref["vel"][live]),
        "stress": rel_l2(gpu["stress"][live], ref["stress"][live]),
        "vol": rel_l2(gpu["vol"][live], ref["vol"][live]),
        "dvol": rel_l2((gpu["vol"] - start["vol"])[live], (ref["vol"] - start["vol"])[live],
                       floor=1e-3 * np.linalg.norm(start["vol"])),
    }
    if h is not None:
        out["off_cells"] = float(np.abs(gpu["pos"][live] - ref["pos"][live]).max() / h) if live.any() else 0.0
    return out


def worst(err, keys):
    return max(err[k] for k in keys)


def cell_mismatch_in_band(gpu, ref, h, band_frac):
    """Particles whose GPU cell differs from the oracle's must lie within
    band_frac * h of a cell face in the oracle's position; returns the count
    of differing cells and the count outside the band."""
    diff = gpu["cell"] != ref["cell"]
    if not diff.any():
        return 0, 0
    pos = ref["pos"][diff] / h
    dist = np.abs(pos - np.round(pos)).min(axis=1)
    return int(diff.sum()), int((dist > band_frac).sum())


def small_column(precision=W.FP32_MIXED, scheme=W.USL):
    """Scaled 3D granular column: same physics and cell size as the 512k
    workload on a 40 x 16 x 24 mesh with a 12^3-cell column (13,824 particles);
    its tiles are partly filled and it has a ragged last tile in x and z."""
    return W.column3d(ncells=(40, 16, 24), col_cells=(12, 12, 12), precision=precision, scheme=scheme,
                      name="granular_column_3d_small")


def max_over_rms(a, b):
    """Largest per-particle error norm over the RMS of the reference's
    per-particle norms.  A fault confined to a few particles (a boundary
    layer, the base-friction nodes) shows here; a relative L2 over all
    particles dilutes it."""
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    rms = float(np.sqrt(np.mean(np.sum(b * b, axis=1)))) if len(b) else 0.0
    e = np.sqrt(np.sum((a - b) ** 2, axis=1)) if len(a) else np.zeros(1)
    return float(e.max() / rms) if rms > 0 else float(e.max())


def per_particle(gpu, ref, start):
    """max_over_rms of displacement (since `start`), velocity and stress over
    the particles live on both sides."""
    live = (gpu["cell"] >= 0) & (ref["cell"] >= 0)
    return {
        "disp": max_over_rms((gpu["pos"] - start["pos"])[live], (ref["pos"] - start["pos"])[live]),
        "vel": max_over_rms(gpu["vel"][live], ref["vel"][live]),
        "stress": max_over_rms(gpu["stress"][live], ref["stress"][live]),
    }


# Resolution of the FP32 cell offset: the offset lies in [-0.5, 0.5) cells, so
# one rounding of it is at most 2^-26 cells; a step rounds it once.
OFFSET_ROUNDING_CELLS = 2.0 ** -26


def disp_excess(gpu, ref, start, h, steps, dim, rel=TOL_RUN_FP32, unit=None):
    """Per-particle displacement error beyond what the FP32 offset can
    resolve: the largest of |d_gpu - d_ref| / (rel * rms(d_ref) + floor)
    over the live particles, with floor = (steps + 1) * 2 * unit h sqrt(dim)
    (the rounding of the initial offset and of every step's, twice over;
    unit = 2^-26 cell for the Cartesian offset).  Values <= 1 pass."""
    unit = OFFSET_ROUNDING_CELLS if unit is None else unit
    live = (gpu["cell"] >= 0) & (ref["cell"] >= 0)
    dg = (gpu["pos"] - start["pos"])[live]
    dr = (ref["pos"] - start["pos"])[live]
    rms = float(np.sqrt(np.mean(np.sum(dr * dr, axis=1)))) if len(dr) else 0.0
    floor = (steps + 1) * 2.0 * unit * h * math.sqrt(dim)
    e = np.sqrt(np.sum((dg - dr) ** 2, axis=1))
    return float(e.max() / (rel * rms + floor)) if len(e) else 0.0


def named_workload(name, precision=W.FP32_MIXED, scheme=W.USL):
    """Workloads the long parity runs use (built the same way in a worker
    process and in the test)."""
    if name == "small_column":
        return small_column(precision=precision, scheme=scheme)
    if name == "slope_1_64":
        wl = W.slope3d(ncells=(200, 50, 50), h=0.2, crest=8.0, plateau=8.5, precision=precision)
        wl.scheme = scheme
        return wl
    if name == "plate_with_hole":
        return W.plate_with_hole(precision=precision, scheme=scheme)
    raise ValueError(name)


def oracle_checkpoints(job):
    """Run the oracle on a named workload from its inputs and snapshot it at
    the given steps (a worker of a spawned process pool: the oracle is
    sequential, so independent runs go to separate cores)."""
    name, scheme, checkpoints = job
    wl = named_workload(name, scheme=scheme)
    o = oracle_from_workload(wl, scheme)
    out = {0: oracle_snapshot(o, wl.dim)}
    done = 0
    for k in sorted(checkpoints):
        st = o.step(k - done)
        done = k
        snap = oracle_snapshot(o, wl.dim)
        snap["status"] = st
        out[k] = snap
    return out


def check_step(gpu, ref, start, h, dim, steps=1):
    """The per-step FP32 bar from an identical state (or a few steps from the
    inputs): position, velocity, stress and volume within TOL_STEP_FP32
    (relative L2); per particle, velocity within 1e-4 and stress within 1e-3
    of the field's RMS; and the displacement of every particle within
    TOL_STEP_FP32 of its RMS plus the offset's rounding (disp_excess).  The
    displacement check is what holds advection to account: positions
    measured from the mesh origin barely move in one step."""
    err = compare(gpu, ref, start, dim)
    assert worst(err, STATE_KEYS) <= TOL_STEP_FP32, err
    pp = per_particle(gpu, ref, start)
    assert pp["vel"] <= 1e-4 and pp["stress"] <= 1e-3, pp
    ex = disp_excess(gpu, ref, start, h, steps, dim, rel=TOL_STEP_FP32)
    assert ex <= 1.0, ex
    return err
