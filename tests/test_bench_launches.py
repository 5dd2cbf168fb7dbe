"""The bench's per-step kernel count (its gpu_launches claim) follows the
step's structure: three binning kernels, then P2G, the nodal update and G2P
(USL), plus the FP64 apex-band kernel when the material has cohesion."""
import dataclasses

import numpy as np

import bench
from paper_1909_13380_gb300 import workloads as W


def _small_column(**kw):
    wl = W.column3d(ncells=(40, 16, 24), col_cells=(4, 4, 4))
    return dataclasses.replace(wl, **kw) if kw else wl


def test_cohesionless_column_launches_six_kernels_per_step():
    wl = _small_column()
    assert wl.material["c"] == 0.0 and wl.coh is None
    assert bench.binning_launches(wl) == 3
    assert bench.apex_launches(wl) == 0


def test_cohesion_adds_the_apex_band_kernel():
    wl = _small_column()
    assert bench.apex_launches(dataclasses.replace(wl, material=dict(wl.material, c=10e3))) == 1
    assert bench.apex_launches(dataclasses.replace(wl, coh=np.full(wl.n, 5e3))) == 1
    # a linear-elastic material never reaches the Mohr-Coulomb return
    el = dataclasses.replace(wl, material=dict(wl.material, model=W.LINEAR_ELASTIC, c=10e3))
    assert bench.apex_launches(el) == 0
