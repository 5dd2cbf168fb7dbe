"""Failure detection of the bounded device wait (no GPU fault involved).

The FP32 tile scan of a mesh past 4095 tiles waits, on the device, for the
prefix each earlier chunk publishes.  The test hook withholds one chunk's
flag, so the chunks after it wait until their (lowered) poll limit runs out:
the step must end, latch MPM_ERR_TIMEOUT for mpm_sync, freeze that mesh
(later steps carry it over and touch nothing else), and leave a fresh mesh
and a mesh stepped alongside it untouched."""
import numpy as np
import pytest

from paper_1909_13380_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - runs only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1909_13380_gb300 import mpm  # noqa: E402


def wide():
    # 120 x 48 x 48 cells: 4320 tiles, the look-back scan over five chunks
    return W.column3d(ncells=(120, 48, 48), col_cells=(12, 12, 12), name="wide_column")


def run(wl, steps):
    with mpm.Simulation(wl) as s:
        s.step(steps)
        snap, st = s.read()
    return snap, st


def test_withheld_scan_flag_times_out_and_freezes_only_that_mesh():
    wl = wide()
    ref5, st = run(wl, 5)
    assert st == mpm.MPM_OK
    bystander = mpm.Simulation(wl)
    with mpm.Simulation(wl) as s:
        s.step(2)
        assert s.sync() == mpm.MPM_OK
        mpm.mpm_set_scan_fault(s.h, 1, 4096)
        s.step(1)
        bystander.step(5)
        assert s.sync() == mpm.MPM_ERR_TIMEOUT
        # frozen: the steps are still enqueued (they carry the mesh over) and
        # report the latched status; nothing faults
        assert mpm.load().mpm_step(s.h, 3) == mpm.MPM_ERR_TIMEOUT
        assert s.sync() == mpm.MPM_ERR_TIMEOUT
        snap, st = s.read()
        assert st == mpm.MPM_ERR_TIMEOUT
        assert np.all(np.isfinite(snap["pos"]))
    # the mesh stepped alongside it and a fresh one are untouched
    got, st = bystander.read()
    bystander.close()
    assert st == mpm.MPM_OK
    for k in ref5:
        assert np.array_equal(got[k], ref5[k]), k
    fresh, st = run(wl, 5)
    assert st == mpm.MPM_OK
    for k in ref5:
        assert np.array_equal(fresh[k], ref5[k]), k


def test_scan_fault_arguments():
    with mpm.Simulation(H.small_column()) as s:
        for bad in ((-2, 10), (0, 0), (0, (1 << 20) + 1)):
            with pytest.raises(mpm.MPMError) as ei:
                mpm.mpm_set_scan_fault(s.h, *bad)
            assert ei.value.status == mpm.MPM_ERR_ARG
        # a mesh scanned by one CTA has no waits: the hook changes nothing
        mpm.mpm_set_scan_fault(s.h, 0, 16)
        s.step(3)
        assert s.sync() == mpm.MPM_OK
