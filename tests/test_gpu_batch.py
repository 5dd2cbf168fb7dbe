"""Batched steps of independent meshes (the serving path): one launch per
phase over all admitted meshes, replayed from a CUDA graph.  Meshes share no
data, so every mesh's state must be bit-identical to stepping it alone --
whatever else is in the batch, and across admissions and evictions."""
import numpy as np
import pytest

from paper_1909_13380_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - runs only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1909_13380_gb300 import mpm  # noqa: E402


def mix():
    """Mixed sizes, dimensions and schemes: small 2D columns of the batched
    workload, a 3D column, and the elastic bar in FP32 (USF)."""
    cols = W.columns2d_batch(count=3, seed=W.SEED_BASE + 33)
    return cols + [W.column2d(6, 8, mesh_cells=(20, 12), name="column2d_small"), H.small_column(),
                   W.elastic_bar(precision=W.FP32_MIXED, scheme=W.USF)]


def alone(wl, steps):
    with mpm.Simulation(wl) as s:
        s.step(steps)
        snap, st = s.read()
    return snap, st


def equal(a, b):
    return all(np.array_equal(a[k], b[k], equal_nan=True) for k in a)


def test_batch_results_equal_alone_runs():
    wls = mix()
    steps = 40
    sims = [mpm.Simulation(w) for w in wls]
    b = mpm.mpm_batch_create()
    try:
        slots = [mpm.mpm_batch_admit(b, s.h) for s in sims]
        assert slots == list(range(len(wls)))
        mpm.mpm_batch_step(b, steps)
        assert mpm.mpm_batch_poll(b, len(wls)) == [mpm.MPM_OK] * len(wls)
        for wl, s in zip(wls, sims):
            snap, st = s.read()
            assert st == mpm.MPM_OK
            ref, _ = alone(wl, steps)
            assert equal(snap, ref), wl.name
    finally:
        mpm.mpm_batch_destroy(b)
        for s in sims:
            s.close()


def test_batch_with_a_mesh_past_the_one_cta_scan():
    # a 16,640-tile mesh (past the one-CTA scan's 4096) sends its whole group
    # through the look-back tile scan over many CTAs; the small mesh beside
    # it must not notice
    wls = [W.column3d(ncells=(260, 64, 64), col_cells=(12, 12, 12), name="column3d_16640_tiles"),
           H.small_column()]
    steps = 30
    sims = [mpm.Simulation(w) for w in wls]
    b = mpm.mpm_batch_create()
    try:
        for s in sims:
            mpm.mpm_batch_admit(b, s.h)
        mpm.mpm_batch_step(b, steps)
        assert mpm.mpm_batch_poll(b, len(wls)) == [mpm.MPM_OK] * len(wls)
        for wl, s in zip(wls, sims):
            snap, st = s.read()
            assert st == mpm.MPM_OK
            ref, _ = alone(wl, steps)
            assert equal(snap, ref), wl.name
    finally:
        mpm.mpm_batch_destroy(b)
        for s in sims:
            s.close()


def test_admission_and_eviction_mid_run():
    wls = mix()[:4]
    sims = [mpm.Simulation(w) for w in wls]
    b = mpm.mpm_batch_create()
    try:
        s0 = mpm.mpm_batch_admit(b, sims[0].h)
        s1 = mpm.mpm_batch_admit(b, sims[1].h)
        mpm.mpm_batch_step(b, 7)                      # 0, 1 at 7 steps
        s2 = mpm.mpm_batch_admit(b, sims[2].h)
        mpm.mpm_batch_step(b, 5)                      # 0, 1 at 12; 2 at 5
        mpm.mpm_batch_evict(b, s1)                    # 1 leaves at 12 and goes on alone
        sims[1].step(3)                               # 1 at 15
        s3 = mpm.mpm_batch_admit(b, sims[3].h)
        assert s3 == s1                               # the freed slot is reused
        mpm.mpm_batch_step(b, 4)                      # 0 at 16, 2 at 9, 3 at 4
        expect = {0: 16, 1: 15, 2: 9, 3: 4}
        for i, s in enumerate(sims):
            snap, st = s.read()
            ref, _ = alone(wls[i], expect[i])
            assert equal(snap, ref), (i, wls[i].name)
        status = mpm.mpm_batch_poll(b, 4)
        assert status[s0] == mpm.MPM_OK and status[s2] == mpm.MPM_OK and status[s3] == mpm.MPM_OK
    finally:
        mpm.mpm_batch_destroy(b)
        for s in sims:
            s.close()


def test_poll_reports_only_the_failing_mesh():
    ok = W.column2d(4, 4, mesh_cells=(16, 10), name="ok")
    pos = np.array([[0.0995, 0.05], [0.05, 0.05]])
    bad = W.Workload(name="leaves", dim=2, ncells=(10, 10, 1), h=0.01, origin=(0, 0, 0), face_bc=(0,) * 6,
                     face_mu=(0,) * 6, gravity=(0, 0, 0), dt=1e-5, scheme=W.USL, precision=W.FP32_MIXED,
                     material=dict(model=0, E=1e3, nu=0.2, rho=1000.0, phi=0, c=0, psi=0), pos=pos,
                     vel=np.array([[200.0, 0.0], [0.0, 0.0]]), vol=np.full(2, 2.5e-5))
    sims = [mpm.Simulation(ok), mpm.Simulation(bad)]
    b = mpm.mpm_batch_create()
    try:
        for s in sims:
            mpm.mpm_batch_admit(b, s.h)
        mpm.mpm_batch_step(b, 5)
        assert mpm.mpm_batch_poll(b, 3) == [mpm.MPM_OK, mpm.MPM_ERR_LEFT_MESH, mpm.MPM_ERR_STATE]
    finally:
        mpm.mpm_batch_destroy(b)
        for s in sims:
            s.close()


def test_footprint_covers_the_allocation():
    wl = W.column3d()
    d = mpm.make_desc(wl.dim, wl.ncells, wl.h, precision=W.FP32_MIXED)
    est = mpm.mpm_footprint(d, wl.n)
    free0 = torch.cuda.mem_get_info()[0]
    with mpm.Simulation(wl) as s:
        s.step(1)
        s.sync()
        used = free0 - torch.cuda.mem_get_info()[0]
    assert est > 0.9 * used


def test_budget_and_slots_refuse_admission_and_leave_the_batch_intact():
    """A batch with a memory budget that holds two of three meshes, then one
    with a single slot: the refused admission returns MPM_ERR_OOM, the mesh
    and the batch are unchanged, and the admitted meshes still step as they
    would alone; an eviction makes room."""
    wls = W.columns2d_batch(count=3, seed=W.SEED_BASE + 35)
    fps = []
    for wl in wls:
        d = mpm.make_desc(wl.dim, wl.ncells, wl.h, precision=W.FP32_MIXED, scheme=wl.scheme)
        fps.append(mpm.mpm_footprint(d, wl.n, False))
    sims = [mpm.Simulation(w) for w in wls]
    steps = 12
    b = mpm.mpm_batch_create(hbm_budget_bytes=sum(fps) - 1, max_slots=8)
    try:
        assert mpm.mpm_batch_admit(b, sims[0].h) == 0
        assert mpm.mpm_batch_admit(b, sims[1].h) == 1
        room, free_slots = mpm.mpm_batch_room(b)
        assert room < fps[2] and free_slots == 6
        with pytest.raises(mpm.MPMError) as ei:
            mpm.mpm_batch_admit(b, sims[2].h)
        assert ei.value.status == mpm.MPM_ERR_OOM
        assert sims[2].sync() == mpm.MPM_OK          # not latched on the refused mesh
        mpm.mpm_batch_step(b, steps)
        status, taken = mpm.mpm_batch_poll(b, 3, with_steps=True)
        assert status == [mpm.MPM_OK, mpm.MPM_OK, mpm.MPM_ERR_STATE] and taken == [steps, steps, -1]
        for i in (0, 1):
            snap, _ = sims[i].read()
            assert equal(snap, alone(wls[i], steps)[0]), i
        mpm.mpm_batch_evict(b, 0)
        assert mpm.mpm_batch_admit(b, sims[2].h) == 0   # the evicted mesh's budget and slot are free again
        mpm.mpm_batch_step(b, steps)
        status, taken = mpm.mpm_batch_poll(b, 2, with_steps=True)
        assert status == [mpm.MPM_OK, mpm.MPM_OK] and taken == [steps, 2 * steps]
        snap, _ = sims[2].read()
        assert equal(snap, alone(wls[2], steps)[0])
        assert mpm.mpm_batch_step_kernels(b) >= 6
    finally:
        mpm.mpm_batch_destroy(b)
    b = mpm.mpm_batch_create(max_slots=1)
    try:
        mpm.mpm_batch_admit(b, sims[0].h)
        with pytest.raises(mpm.MPMError) as ei:
            mpm.mpm_batch_admit(b, sims[1].h)
        assert ei.value.status == mpm.MPM_ERR_OOM
    finally:
        mpm.mpm_batch_destroy(b)
        for s in sims:
            s.close()
