"""The serving loop on the GPU: requests of mixed kinds and sizes arrive
while others run, are admitted and batched, and each result is bit-identical
to running the same request alone; the one-at-a-time FP64 engine serves the
same stream within the FP32-vs-FP64 tolerance."""
import numpy as np
import pytest

from paper_1909_13380_gb300 import serve
from paper_1909_13380_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - runs only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1909_13380_gb300 import mpm  # noqa: E402


def stream(count=10):
    reqs = W.serving_requests(count=count, rate=400.0, n_range=(3e3, 4e4), steps_range=(8, 60), step_scale=1.0,
                              seed=W.SEED_BASE + 41)
    return reqs, [r.workload() for r in reqs]


def alone(wl, steps, precision=W.FP32_MIXED):
    with mpm.Simulation(wl, precision=precision) as s:
        s.step(steps)
        snap, st = s.read(serve.RESULT_FIELDS)
    return snap, st


def test_batched_serving_equals_alone_runs():
    reqs, wls = stream()
    eng = serve.GpuEngine(batched=True)
    try:
        done, lat, total = serve.Server(eng, chunk=5, keep_results=True).run(reqs, wls)
    finally:
        eng.shutdown()
    assert sorted(f.rid for f in done) == list(range(len(reqs)))
    assert len({r.kind for r in reqs}) >= 3
    # requests overlapped: some were admitted before an earlier one finished
    fin = {f.rid: f.finished for f in done}
    assert any(f.admitted < fin[g.rid] and g.rid < f.rid for f in done for g in done)
    for f in done:
        assert f.status == mpm.MPM_OK, (f.rid, f.kind)
        ref, st = alone(wls[f.rid], reqs[f.rid].steps)
        assert st == mpm.MPM_OK
        for k in serve.RESULT_FIELDS:
            assert np.array_equal(f.result[k], ref[k]), (f.rid, f.kind, k)
    rep = serve.report(done, lat, total)
    assert rep["step_ms"]["p99"] >= rep["step_ms"]["p50"] > 0
    assert eng.h2d > 0 and eng.d2h > 0


def test_fp64_one_at_a_time_matches_fp32_batched():
    reqs, wls = stream(count=4)
    res = {}
    for name, eng in (("fp32", serve.GpuEngine(batched=True)),
                      ("fp64", serve.GpuEngine(precision=W.FP64_PLAIN, batched=False))):
        try:
            done, lat, total = serve.Server(eng, chunk=5, keep_results=True).run(reqs, wls)
        finally:
            eng.shutdown()
        assert all(f.status == mpm.MPM_OK for f in done)
        res[name] = {f.rid: f.result for f in done}
    for i in range(len(reqs)):
        wl, steps = wls[i], reqs[i].steps
        live = np.zeros(wl.n, np.int64)
        g = {"pos": res["fp32"][i]["pos"], "cell": live}
        r = {"pos": res["fp64"][i]["pos"], "cell": live}
        # displacements from the request's inputs: within 1e-3 of their RMS per
        # particle, plus the FP32 offset's rounding over the steps taken
        assert H.disp_excess(g, r, {"pos": wl.pos}, wl.h, steps, wl.dim) <= 1.0, i
        for k in ("vel", "stress"):
            a, b = res["fp32"][i][k], res["fp64"][i][k]
            assert H.rel_l2(a, b) <= H.TOL_RUN_FP32, (i, k)
            assert H.max_over_rms(a, b) <= 1e-2, (i, k)
