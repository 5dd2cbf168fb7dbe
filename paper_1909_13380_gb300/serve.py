"""Serving loop: continuous batching of independent explicit MPM simulations.

Requests (a mesh, its particles and a step count) arrive over time.  Each is
admitted as soon as the device has memory for it (its footprint against the
free HBM), its state stays resident, and every admitted simulation advances
in the same batched steps -- one launch per phase over all of them, replayed
from a CUDA graph -- until it has taken its steps; then its result (particle
positions, velocities and stresses) is read back and its memory released.
Admission happens between chunks of batched steps, so requests that arrive
while others run join them without waiting for the batch to drain, and the
upload of a newly arrived request overlaps the running chunk.

The paper runs one simulation per process (CODE OVERVIEW, DATA STRUCTURES);
this loop is the serving form of the same explicit step.  All arithmetic runs
in the CUDA library; this module only schedules.

`Server.run` is written against a small engine interface (`GpuEngine` below)
so that its scheduling can be tested on the host with a fake engine.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np

from . import workloads as W

RESULT_FIELDS = ("pos", "vel", "stress")
ERR_OOM = -2          # MPM_ERR_OOM: the request does not fit the free device memory


@dataclass
class Finished:
    rid: int
    kind: str
    n: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    status: int
    result: dict | None = None

    @property
    def e2e(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    rid: int
    sim: object
    remaining: int
    admitted: float


class GpuEngine:
    """The CUDA library behind the serving loop.  `batched` selects
    continuous batching (one batch over every admitted FP32 simulation) or
    one simulation at a time (any precision).

    The batch owns admission: it is created with a device-memory budget (the
    free HBM at start, less a reserve) and a slot count, and the library
    refuses a mesh (MPM_ERR_OOM) whose footprint exceeds what the budget has
    left.  Meshes created for the next admission point (their upload overlaps
    the running chunk) hold memory before they are admitted, so the room the
    loop sees is the batch's room less their footprints."""

    def __init__(self, precision=W.FP32_MIXED, batched=True, reserve_bytes=2 << 30, max_slots=4096):
        import torch

        from . import mpm
        self.torch, self.mpm = torch, mpm
        self.precision = precision
        self.batched = batched
        self.reserve = int(reserve_bytes)
        self.side = torch.cuda.Stream()          # uploads and result reads (and unbatched steps)
        self.bstream = torch.cuda.Stream()       # batched steps
        self.batch = None
        if batched:
            budget = max(1, int(torch.cuda.mem_get_info()[0]) - self.reserve)
            self.batch = mpm.mpm_batch_create(self.bstream.cuda_stream, hbm_budget_bytes=budget,
                                              max_slots=max_slots)
        self.staged = {}                         # id(sim) -> footprint of meshes created, not yet admitted
        self.h2d = 0
        self.d2h = 0

    def footprint(self, wl) -> int:
        d = self.mpm.make_desc(wl.dim, wl.ncells, wl.h, precision=self.precision, scheme=wl.scheme)
        return self.mpm.mpm_footprint(d, wl.n, wl.coh is not None)

    def free_bytes(self) -> int:
        if self.batched:
            room, slots = self.mpm.mpm_batch_room(self.batch)
            return room - sum(self.staged.values()) if slots > len(self.staged) else -1
        return int(self.torch.cuda.mem_get_info()[0]) - self.reserve

    def create(self, wl):
        sim = self.mpm.Simulation(wl, precision=self.precision, stream=self.side.cuda_stream)
        self.h2d += wl.pos.nbytes + wl.vel.nbytes + wl.vol.nbytes + (wl.coh.nbytes if wl.coh is not None else 0)
        if self.batched:
            self.staged[id(sim)] = self.footprint(wl)
        return sim

    def admit(self, sim):
        """The slot of the admitted simulation, or None when the batch
        refuses it (MPM_ERR_OOM: no slot or budget left yet)."""
        try:
            slot = self.mpm.mpm_batch_admit(self.batch, sim.h)
        except self.mpm.MPMError as e:
            if e.status == self.mpm.MPM_ERR_OOM:
                return None
            raise
        self.staged.pop(id(sim), None)
        return slot

    def evict(self, slot: int):
        self.mpm.mpm_batch_evict(self.batch, slot)

    def launch(self, k: int, sims):
        """Enqueue k steps of the admitted simulations (batched) or of the
        one simulation given; returns a handle for `wait`."""
        torch = self.torch
        st = self.bstream if self.batched else self.side
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        if self.batched:
            self.mpm.mpm_batch_step(self.batch, k)
        else:
            for s in sims:
                s.step(k)
        e1.record(st)
        return (e0, e1)

    def wait(self, handle, nslots: int, sims):
        """Wait for a launch; returns (device ms, per-slot status)."""
        e0, e1 = handle
        e1.synchronize()
        if self.batched:
            status = self.mpm.mpm_batch_poll(self.batch, nslots)
        else:
            status = [s.sync() for s in sims]
        return e0.elapsed_time(e1), status

    def read(self, sim):
        snap, st = sim.read(RESULT_FIELDS)
        self.d2h += sum(a.nbytes for a in snap.values())
        return snap, st

    def close(self, sim):
        sim.close()

    def shutdown(self):
        if self.batch is not None:
            self.mpm.mpm_batch_destroy(self.batch)
            self.batch = None


class Server:
    """Continuous batching over an engine.  chunk: batched steps between two
    admission points; keep_results: return each request's result arrays."""

    def __init__(self, engine, chunk=16, keep_results=False, max_active=4096, clock=time.perf_counter,
                 sleep=time.sleep):
        self.eng = engine
        self.chunk = int(chunk)
        self.keep = keep_results
        self.max_active = max_active
        self.clock = clock
        self.sleep = sleep

    def run(self, requests, workloads):
        """Serve `requests` (sorted by arrival) whose inputs are `workloads`
        (prepared by the caller: the client builds a request before it
        arrives).  Returns (finished requests, per-step latencies in ms with
        their step counts, session seconds)."""
        eng = self.eng
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        queue = collections.deque()
        active: dict[int, _Active] = {}
        single: list[_Active] = []        # one-at-a-time engines
        done: list[Finished] = []
        lat: list[tuple[float, int]] = []
        nxt = 0
        t0 = self.clock()
        nslots = 0
        nparts: dict[int, int] = {}
        # a workload source may drop a request's host arrays once it is on
        # the device (see RequestStream)
        release = getattr(workloads, "release", lambda i: None)

        def now():
            return self.clock() - t0

        def arrivals():
            nonlocal nxt
            while nxt < len(order) and requests[order[nxt]].arrival <= now():
                queue.append(order[nxt])
                nxt += 1

        def admit_ready(staged):
            # FIFO by free memory: the head waits until it fits
            while queue and len(active) + len(staged) + len(single) < self.max_active:
                if not eng.batched and (single or staged):
                    break
                i = queue[0]
                if eng.footprint(workloads[i]) > eng.free_bytes():
                    if active or single or staged:
                        break                     # wait for memory to free up
                    queue.popleft()               # larger than the whole free device
                    r = requests[i]
                    t = now()
                    done.append(Finished(i, r.kind, workloads[i].n, r.steps, r.arrival, t, t, ERR_OOM))
                    release(i)
                    continue
                queue.popleft()
                nparts[i] = workloads[i].n
                staged.append((i, eng.create(workloads[i]), now()))
                release(i)                        # the inputs are on the device now

        def finish(a: _Active, status: int):
            snap = None
            if self.keep or status == 0:
                snap, st = eng.read(a.sim)
                status = status or st
            eng.close(a.sim)
            r = requests[a.rid]
            done.append(Finished(a.rid, r.kind, nparts[a.rid], r.steps, r.arrival, a.admitted, now(),
                                 status, snap if self.keep else None))

        staged: list = []
        while nxt < len(order) or queue or active or single or staged:
            arrivals()
            admit_ready(staged)
            refused = []
            for i, sim, t_adm in staged:
                a = _Active(i, sim, requests[i].steps, t_adm)
                if eng.batched:
                    slot = eng.admit(sim)
                    if slot is None:              # the batch has no room yet: admit it later
                        refused.append((i, sim, t_adm))
                        continue
                    active[slot] = a
                    nslots = max(nslots, slot + 1)
                else:
                    single.append(a)
            staged = refused
            running = list(active.values()) if eng.batched else single
            if not running:
                if nxt < len(order):
                    self.sleep(max(0.0, requests[order[nxt]].arrival - now()))
                continue
            k = min(self.chunk, min(a.remaining for a in running))
            h = eng.launch(k, [a.sim for a in running])
            # arrivals during the chunk are uploaded while it runs
            arrivals()
            admit_ready(staged)
            ms, status = eng.wait(h, nslots, [a.sim for a in running])
            lat.append((ms / k, k))
            if eng.batched:
                for slot in list(active):
                    a = active[slot]
                    a.remaining -= k
                    st = status[slot]
                    if a.remaining == 0 or st != 0:
                        eng.evict(slot)
                        del active[slot]
                        finish(a, st)
            else:
                a = single[0]
                a.remaining -= k
                if a.remaining == 0 or status[0] != 0:
                    single.pop(0)
                    finish(a, status[0])
        return done, lat, now()


class RequestStream:
    """Workloads of a request stream built on a background thread in arrival
    order, at most `ahead` requests before they are consumed (a client that
    prepares its request before sending it), and dropped once the server has
    put them on the device -- so a long session does not hold every
    request's particle arrays in host memory at once.  `build(request)`
    returns the workload."""

    def __init__(self, requests, build, ahead=8):
        import threading
        self.reqs = requests
        self.build = build
        self.ahead = ahead
        self.order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        self.pos = {i: k for k, i in enumerate(self.order)}
        self.ready: dict[int, object] = {}
        self.consumed = 0                 # requests released so far
        self.cv = threading.Condition()
        self.stop = False
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def _run(self):
        for k, i in enumerate(self.order):
            with self.cv:
                while not self.stop and k >= self.consumed + self.ahead:
                    self.cv.wait()
                if self.stop:
                    return
            wl = self.build(self.reqs[i])
            with self.cv:
                self.ready[i] = wl
                self.cv.notify_all()

    def __getitem__(self, i):
        with self.cv:
            while i not in self.ready:
                self.cv.wait()
            return self.ready[i]

    def __len__(self):
        return len(self.reqs)

    def release(self, i):
        with self.cv:
            if self.ready.pop(i, None) is not None:
                self.consumed += 1
                self.cv.notify_all()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.thread.join(timeout=60)


def percentiles(values, weights=None):
    v = np.asarray(values, np.float64)
    if v.size == 0:
        return {"p50": None, "p99": None, "mean": None}
    if weights is not None:
        v = np.repeat(v, np.asarray(weights, np.int64))
    return {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)), "mean": float(v.mean())}


def report(done, lat, session_s):
    """Summary of a session: throughput, p50 / p99 latencies, and the
    utilisation (device time of the steps over the session time)."""
    ps = sum(f.n * f.steps for f in done)
    busy = sum(ms * k for ms, k in lat) * 1e-3
    return {
        "requests": len(done),
        "failed": sum(1 for f in done if f.status != 0),
        "particle_steps": int(ps),
        "session_s": session_s,
        "particle_steps_per_s": ps / session_s if session_s > 0 else None,
        "step_ms": percentiles([x for x, _ in lat], [k for _, k in lat]),
        "e2e_s": percentiles([f.e2e for f in done]),
        "queue_s": percentiles([f.admitted - f.arrival for f in done]),
        "gpu_busy_s": busy,
        "utilisation": busy / session_s if session_s > 0 else None,
    }
