"""Parity at the benchmark's full size: the 63,875,200-particle 3D slope
(800 x 200 x 200 cells) stepped through the C-ABI exactly as the benchmark
times it (one mesh, FP32 mixed USL, the step graph on a stream of its own),
checked against the oracle on a sampled patch.

A step's nodal values at a node depend only on the particles of the cells
around it, so one step of the particles of a patch of cells needs only the
patch and a halo of cells around it.  After 3000 steps (the benchmark's
timed window starts at 1000; by 3000 the stress wave from the fixed base
has crossed the slope) the GPU state of the particles in an 8 x 8 x 8 patch
at the slope's toe on the base plus a halo of 2 cells (none below the base)
goes to an oracle mesh of that box, whose bottom is the base, fixed; one
oracle step then gives, for the particles of the patch, what one more GPU
step must give within the per-step FP32 bar.  The patch holds the fixed
base, cohesive Mohr-Coulomb material under gravity and the tile crossings of
the settling slope.  Properties that hold at any
size are checked over the whole mesh: mass conserved exactly, every
particle still in the mesh, and the binning a stable sort of the keys."""
import numpy as np
import pytest

import oracle
from paper_1909_13380_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected only with -m gpu on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

import ctypes as C  # noqa: E402

from paper_1909_13380_gb300 import mpm  # noqa: E402

PATCH_LO, PATCH_N, HALO = (300, 96, 2), 8, 2   # at the toe (x 15-15.4 m), 0.1-0.5 m above the base
ADVANCE = 3000


def patch_sets(cell, nc):
    """Particles in the patch and halo box, and those in the patch itself."""
    c = np.asarray(cell)
    ix, iy, iz = c % nc[0], (c // nc[0]) % nc[1], c // (nc[0] * nc[1])
    lo = np.array(PATCH_LO)
    inb = np.ones(len(c), bool)
    inp = np.ones(len(c), bool)
    for a, v in enumerate((ix, iy, iz)):
        inb &= (v >= lo[a] - HALO) & (v < lo[a] + PATCH_N + HALO)
        inp &= (v >= lo[a]) & (v < lo[a] + PATCH_N)
    inb &= c >= 0
    return np.nonzero(inb)[0], inp


def read_subset(sim, idx, fields):
    out = {}
    for f in fields:   # one field at a time: the whole mesh's arrays are large
        snap, st = sim.read((f,))
        assert st == mpm.MPM_OK
        out[f] = np.array(snap[f][idx])
        del snap
    return out


def test_slope_64m_patch_step_against_the_oracle():
    wl = W.slope3d()
    assert wl.n == 63_875_200
    stream = torch.cuda.Stream()
    sim = mpm.Simulation(wl, stream=C.c_void_p(stream.cuda_stream))
    try:
        m0 = sim.conservation()[0]["mass"]
        with torch.cuda.stream(stream):
            for _ in range(ADVANCE):
                sim.step(1)
        stream.synchronize()
        assert sim.sync() == mpm.MPM_OK
        # whole-mesh properties
        cons, st = sim.conservation()
        assert st == mpm.MPM_OK and cons["alive"] == wl.n and cons["mass"] == m0
        # the binning is the stable sort of the keys (sampled pairs of neighbours in key order)
        key, perm, _ = sim.binning()
        q = np.arange(0, wl.n - 1, 997)
        ka, kb = key[perm[q]], key[perm[q + 1]]
        assert np.all((ka < kb) | ((ka == kb) & (perm[q] < perm[q + 1])))
        del key, perm
        # the patch state at step ADVANCE
        cell0 = sim.read(("cell",))[0]["cell"]
        idx, _ = patch_sets(cell0, wl.ncells)
        del cell0
        fields = ("pos", "vel", "stress", "strain", "vol", "epsp", "cell")
        s0 = read_subset(sim, idx, fields)
        with torch.cuda.stream(stream):
            sim.step(1)
        stream.synchronize()
        assert sim.sync() == mpm.MPM_OK
        s1 = read_subset(sim, idx, fields)
    finally:
        sim.close()
    inner = patch_sets(s0["cell"], wl.ncells)[1]
    assert inner.sum() > 2000 and len(idx) > inner.sum()
    # the oracle on the patch box, from the GPU state (mass from the inputs)
    lo = np.array(PATCH_LO) - HALO
    assert lo[2] == 0   # the box's bottom face is the slope's fixed base
    bc = [W.FREE] * 6
    bc[4] = wl.face_bc[4]
    box = oracle.Mesh(dim=3, n=(PATCH_N + 2 * HALO,) * 3, h=wl.h, origin=tuple(lo * wl.h), g=wl.gravity,
                      dt=wl.dt, scheme=W.USL, face_bc=tuple(bc))
    st = oracle.State.create(s0["pos"], s0["vel"], wl.vol[idx], wl.material["rho"], coh=wl.coh[idx])
    st.sig[:] = s0["stress"]
    st.eps[:] = s0["strain"]
    st.vol[:] = s0["vol"]
    st.epsp[:] = s0["epsp"]
    o = oracle.Oracle(box, oracle.Material(**wl.material), st)
    assert o.step(1) == oracle.OK
    live = {"cell": np.where(inner, 0, -1)}
    g1 = {**{k: s1[k] for k in ("pos", "vel", "stress", "vol")}, **live}
    r1 = {"pos": st.x[:, :3].copy(), "vel": st.v[:, :3].copy(), "stress": st.sig.copy(), "vol": st.vol.copy(),
          **live}
    start = {"pos": s0["pos"], "vol": s0["vol"]}
    H.check_step(g1, r1, start, wl.h, 3)
    # the patch does move: some particles change cell in the step, stresses are non-trivial
    assert np.abs(s1["pos"] - s0["pos"])[inner].max() > 0.0
    assert np.abs(s1["stress"][inner]).max() > 1e3
