"""Scheduling of the serving loop, on the host with a fake engine: every
request takes exactly its steps, admission is first-come first-served by free
memory, memory is never over-committed, batched requests overlap and the
one-at-a-time engine never runs two at once."""
import numpy as np
import pytest

from paper_1909_13380_gb300 import serve
from paper_1909_13380_gb300 import workloads as W


class FakeSim:
    def __init__(self, wl):
        self.wl, self.steps, self.closed = wl, 0, False


class FakeEngine:
    """Memory: footprint = 100 bytes per particle out of `capacity`; a
    batched step takes 1 us per 1000 resident particles + 2 ms (small
    meshes are latency-bound, so one launch over many of them pays off)."""

    def __init__(self, batched, capacity, clock):
        self.batched, self.capacity, self.clock = batched, capacity, clock
        self.slots, self.resident, self.log = {}, 0, []
        self.max_resident = 0
        self.max_running = 0

    def footprint(self, wl):
        return 100 * wl.n

    def free_bytes(self):
        return self.capacity - self.resident

    def create(self, wl):
        self.resident += self.footprint(wl)
        self.max_resident = max(self.max_resident, self.resident)
        return FakeSim(wl)

    def admit(self, sim):
        s = next(i for i in range(len(self.slots) + 1) if i not in self.slots)
        self.slots[s] = sim
        return s

    def evict(self, slot):
        del self.slots[slot]

    def launch(self, k, sims):
        for s in sims:
            assert not s.closed
            s.steps += k
            assert s.steps <= s.wl.steps
        self.max_running = max(self.max_running, len(sims))
        ms = k * (2.0 + 1e-3 * sum(s.wl.n for s in sims) / 1000)
        return (ms, len(sims))

    def wait(self, h, nslots, sims):
        ms, _ = h
        self.clock[0] += ms * 1e-3
        if self.batched:
            return ms, [0 if i in self.slots else -5 for i in range(nslots)]
        return ms, [0] * len(sims)

    def read(self, sim):
        return {"steps": sim.steps}, 0

    def close(self, sim):
        sim.closed = True
        self.resident -= self.footprint(sim.wl)


class TinyWl:
    def __init__(self, n, steps):
        self.n, self.steps = n, steps


def session(batched, capacity=10_000_000, count=40, chunk=8):
    reqs = W.serving_requests(count=count, rate=50.0, n_range=(1e3, 5e4), steps_range=(5, 200), step_scale=1.0)
    wls = [TinyWl(r.n_target, r.steps) for r in reqs]
    clock = [0.0]

    def sleep(dt):
        clock[0] += dt

    eng = FakeEngine(batched, capacity, clock)
    srv = serve.Server(eng, chunk=chunk, keep_results=True, clock=lambda: clock[0], sleep=sleep)
    done, lat, total = srv.run(reqs, wls)
    return reqs, wls, eng, done, lat, total


@pytest.mark.parametrize("batched", [True, False])
def test_every_request_takes_exactly_its_steps(batched):
    reqs, wls, eng, done, lat, total = session(batched)
    assert sorted(f.rid for f in done) == list(range(len(reqs)))
    for f in done:
        assert f.result["steps"] == reqs[f.rid].steps
        assert f.status == 0
        assert f.arrival <= f.admitted <= f.finished
    assert eng.resident == 0
    assert sum(k for _, k in lat) >= max(r.steps for r in reqs)


def test_batched_overlaps_and_sequential_does_not():
    _, _, eb, done_b, _, tb = session(True)
    _, _, es, done_s, _, ts = session(False)
    assert eb.max_running > 1
    assert es.max_running == 1
    # batching finishes the same work sooner
    assert tb < ts
    e2e_b = serve.percentiles([f.e2e for f in done_b])
    e2e_s = serve.percentiles([f.e2e for f in done_s])
    assert e2e_b["p99"] < e2e_s["p99"]


def test_admission_is_fifo_and_bounded_by_memory():
    cap = 6_000_000       # room for a few of the larger requests at a time
    reqs, wls, eng, done, _, _ = session(True, capacity=cap)
    assert eng.max_resident <= cap
    by_arrival = sorted(done, key=lambda f: (reqs[f.rid].arrival, f.rid))
    adm = [f.admitted for f in by_arrival]
    assert adm == sorted(adm)
    # memory bound: some requests had to wait in the queue
    assert any(f.admitted > f.arrival for f in done)


class SlotLimitedEngine(FakeEngine):
    """A batch with two slots: admission beyond them is refused (the library
    answers MPM_ERR_OOM, the engine returns None) and must be retried."""

    def admit(self, sim):
        if len(self.slots) >= 2:
            self.refused = getattr(self, "refused", 0) + 1
            return None
        return super().admit(sim)


def test_refused_admission_is_retried_after_an_eviction():
    reqs = W.serving_requests(count=30, rate=200.0, n_range=(1e3, 5e4), steps_range=(5, 200), step_scale=1.0)
    wls = [TinyWl(r.n_target, r.steps) for r in reqs]
    clock = [0.0]

    def sleep(dt):
        clock[0] += dt

    eng = SlotLimitedEngine(True, 10_000_000, clock)
    done, lat, total = serve.Server(eng, chunk=8, keep_results=True, clock=lambda: clock[0],
                                    sleep=sleep).run(reqs, wls)
    assert sorted(f.rid for f in done) == list(range(len(reqs)))
    assert all(f.result["steps"] == reqs[f.rid].steps and f.status == 0 for f in done)
    assert eng.refused > 0 and eng.max_running <= 2
    assert eng.resident == 0


def test_percentiles_weight_steps():
    p = serve.percentiles([1.0, 10.0], [99, 1])
    assert p["p50"] == 1.0
    assert 1.0 <= p["p99"] <= 10.0
    assert abs(p["mean"] - (99 + 10) / 100) < 1e-12
    assert serve.percentiles([])["p50"] is None


def test_request_generators_hit_their_sizes():
    for kind in W.REQUEST_KINDS:
        for n in (2e4, 2e5):
            wl = W.request_workload(kind, n, seed=7, steps=3)
            assert 0.7 * n < wl.n < 1.3 * n, (kind, n, wl.n)
            assert wl.pos.shape == (wl.n, wl.dim)
            # particles strictly inside the mesh
            for k in range(wl.dim):
                assert wl.pos[:, k].min() > 0 and wl.pos[:, k].max() < wl.ncells[k] * wl.h


def test_request_larger_than_the_device_is_rejected():
    reqs, wls, eng, done, _, _ = session(True, capacity=1_000_000)
    big = {f.rid for f in done if f.status == serve.ERR_OOM}
    assert big == {i for i, w in enumerate(wls) if 100 * w.n > 1_000_000}
    assert len(big) > 0
    assert all(f.status == 0 for f in done if f.rid not in big)
    assert sorted(f.rid for f in done) == list(range(len(reqs)))


def test_utilisation_is_device_time_over_session():
    reqs, wls, eng, done, lat, total = session(True)
    rep = serve.report(done, lat, total)
    busy = sum(ms * k for ms, k in lat) * 1e-3
    assert rep["gpu_busy_s"] == busy
    assert 0.0 < rep["utilisation"] <= 1.0 + 1e-12


def test_request_stream_builds_ahead_and_drops_released():
    reqs = W.serving_requests(count=30, rate=50.0, n_range=(1e3, 5e4), steps_range=(5, 200), step_scale=1.0)
    built = []

    def build(r):
        built.append(r.rid)
        return TinyWl(r.n_target, r.steps)

    stream = serve.RequestStream(reqs, build, ahead=4)
    clock = [0.0]

    def sleep(dt):
        clock[0] += dt

    eng = FakeEngine(True, 10_000_000, clock)
    try:
        done, lat, total = serve.Server(eng, chunk=8, keep_results=True, clock=lambda: clock[0],
                                        sleep=sleep).run(reqs, stream)
    finally:
        stream.close()
    assert sorted(f.rid for f in done) == list(range(len(reqs)))
    assert all(f.result["steps"] == reqs[f.rid].steps for f in done)
    assert all(f.n == reqs[f.rid].n_target for f in done)
    assert sorted(built) == list(range(len(reqs)))
    assert len(stream.ready) == 0          # every request's arrays were dropped after admission
