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
