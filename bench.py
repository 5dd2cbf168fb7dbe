#!/usr/bin/env python
"""Throughput of the explicit MPM step on GB300.

Default workload: the large 3D slope -- 800 x 200 x 200 hexahedra of 0.05 m,
a 45-degree slope section filled with 8 particles per cell (63.9M particles),
Mohr-Coulomb with lognormal per-cell cohesion, fixed base, roller sides, FP32
mixed precision, USL.  A "step" is one explicit MPM time step of the whole
path (binning, P2G, nodal solve with boundary conditions, G2P with the stress
update and relocation, and the FP64 apex-band return).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload slope|column3d|...] [--advance A] [--detail-out PATH]

Timing: A untimed steps bring the run into its middle (the slope workload
runs 2000 steps; A = 1000 by default), then W untimed warm-up steps, then K
steps each bracketed by CUDA events on the library's stream, with a 256 MiB
buffer written between steps (the L2 flushed); max over ranks.  Prints one
JSON line (rank 0).  With N > 1 (torchrun) every rank runs an independent
replica of the workload on its own GPU (replicas only: the path has no
cross-instance exchange), so value = N x per-rank work / max time ("weak"
scaling).

Beside the headline the line carries the dominant kernel's and the whole
step's HBM roofline (with the plain FP64 GPU step on the same workload), the
other update order (USF), an end-to-end run through the C-ABI from pinned
host buffers ("e2e"), the FP64 CPU oracle on a bounded sample
("cpu_baseline") and the FP32 error against it after enough steps for the
displacements to stand above the offset's resolution ("accuracy"), and short
summaries of 256 batched 2D columns ("batched") and of a serving session
("serving").  --detail-out writes the full detail of these as JSON.

--impl reference times the FP64 CPU oracle (the parity reference) on the
host cores on a bounded sample of the same workload and metric.
"""
from __future__ import annotations

import argparse
import dataclasses
import ctypes as C
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1909_13380_gb300 import workloads as W  # noqa: E402

METRIC = "particle-steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# ncu DRAM traffic summaries by workload: (file, particles it was taken on)
TRAFFIC_FILES = {
    "slope_1_64": (os.path.join(ROOT, "profiles", "dram_traffic_slope3d_1m.txt"), 1000000),
    "slope": (os.path.join(ROOT, "profiles", "dram_traffic_slope3d_1m.txt"), 1000000),
}
KERNEL_SRC = os.path.join(ROOT, "paper_1909_13380_gb300", "csrc", "mpm_fp32.cu")


def make_workload(name: str):
    if name == "slope":
        return W.slope3d()
    if name == "column3d":
        return W.column3d()
    if name == "column3d_small":
        return W.column3d(ncells=(40, 16, 24), col_cells=(12, 12, 12))
    if name == "bar":
        return W.elastic_bar(precision=W.FP32_MIXED)
    if name == "slope_1_64":
        return W.slope3d(ncells=(200, 50, 50), h=0.2, crest=8.0, plateau=8.5)
    if name == "slope_slab":
        return slope_slab()
    raise SystemExit(f"unknown workload {name}")


def slope_slab():
    """The bounded CPU sample of the slope: the same cell size (0.05 m),
    8 particles per cell, material, lognormal cohesion and walls, on a 2 m
    slope section four cells wide (roller sides, so a slab of the extruded
    slope); 76,800 particles."""
    wl = W.slope3d(ncells=(160, 4, 48), h=0.05, crest=2.0, plateau=2.0)
    wl.name = "slope_3d_slab_160x4x48_crest2m"
    return wl


# The CPU sample of each workload (the oracle cannot run the full slope:
# one oracle step of its 63.9M particles takes about a minute on one core).
CPU_SAMPLE = {"slope": "slope_slab", "slope_1_64": "slope_1_64", "column3d": "column3d",
              "column3d_small": "column3d_small", "bar": "bar", "slope_slab": "slope_slab"}


# Algorithmic bytes per particle (what the method must move once: each
# particle word read once and each mutable word written once, plus the
# share of node traffic), FP32 mixed path.
def algorithmic_bytes(dim: int, coh: bool):
    ns = 6 if dim == 3 else 4
    read = 4 + 4 * dim + 4 * dim + 4 * ns + 4 * ns + 12 + (4 if coh else 0)   # cell, off, v, sig, eps, m, V, epsp
    write = read - 4 - (4 if coh else 0)                                      # all but m (and coh)
    nodes_per_particle = 0.15 if dim == 3 else 1.3 / 4
    box = nodes_per_particle * 4 * (1 + 2 * dim)       # a tile's node box of P2G sums, per particle
    p2g = 4 + 4 * dim + 4 * dim + 4 * ns + 8 + box
    g2p = read + write + nodes_per_particle * 4 * 2 * dim
    step = (212 if dim == 3 else 174) + (4 if coh else 0)
    return {"p2g": p2g, "g2p": g2p, "step": step}


# The kernel behind each timed phase.
KERNEL_NAMES = {"p2g": "p2g_tile", "g2p": "g2p"}


def load_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash() -> str:
    with open(KERNEL_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def load_traffic(kernel: str, workload: str, n: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of the
    workload, if it was taken on the current kernel source (else None).  The
    64M-particle slope is too large to capture under the profiling size rule:
    its figure is the 1M-particle slope's scaled by the particle count (the
    traffic is per particle).  Returns (bytes, source) or (None, None)."""
    if workload not in TRAFFIC_FILES:
        return None, None
    path, n_file = TRAFFIC_FILES[workload]
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_hash():
            return None, None
        b = float(kv[f"{kernel}_dram_bytes_per_launch"])
        src = os.path.relpath(path, ROOT)
        if n != n_file:
            b *= n / n_file
            src += f" (scaled by {n}/{n_file} particles)"
        return b, src
    except Exception:
        return None, None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _oracle_replica(args):
    """One replica of the oracle (a spawned process): the named workload's
    first steps until the time budget; returns (particles, steps, seconds)."""
    name, budget_s, max_steps = args
    import oracle
    wl = make_workload(name)
    o = oracle.from_workload(wl)
    t0 = time.perf_counter()
    k = 0
    while k < max_steps:
        o.step(1)
        k += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return wl.n, k, time.perf_counter() - t0


def cpu_oracle_all_cores(name: str, budget_s: float, max_steps: int):
    """The oracle on every host core: one independent replica per core (the
    oracle is sequential by design), started with spawn; aggregate
    particle-steps/s = all replicas' particle-steps / the slowest replica's
    time.  Returns (rate, cores, steps per replica)."""
    import multiprocessing as mp
    cores = max(1, min(os.cpu_count() or 1, 64))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_replica, [(name, budget_s, max_steps)] * cores)
    total = sum(n * k for n, k, _ in res)
    return total / max(dt for _, _, dt in res), cores, [k for _, k, _ in res]


def _rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


def _max_over_rms(a, b):
    """Largest per-particle error norm over the RMS of the reference's
    per-particle norms (a fault confined to a few particles shows here,
    where a relative L2 over all of them dilutes it)."""
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    rms = float(np.sqrt(np.mean(np.sum(b * b, axis=1))))
    e = np.sqrt(np.sum((a - b) ** 2, axis=1))
    return float(e.max() / rms) if rms > 0 else float(e.max())


def cpu_leg(wl_name, budget_s, max_steps, sptr):
    """The CPU baseline: the FP64 oracle on the workload's bounded sample,
    one thread (its state after the timed steps also gives the FP32 and FP64
    GPU error on that sample), then one replica per host core."""
    import oracle
    from paper_1909_13380_gb300 import mpm
    name = CPU_SAMPLE[wl_name]
    cwl = make_workload(name)
    o = oracle.from_workload(cwl)
    t0 = time.perf_counter()
    k = 0
    while k < max_steps:
        o.step(1)
        k += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    rate = cwl.n * k / dt
    # accuracy of both GPU precisions against the oracle's k steps
    d = cwl.dim
    st = o.state
    cells = o.cells()
    nc = o.mesh.n
    ref_cell = np.where(cells[:, 0] >= 0, cells[:, 0] + nc[0] * (cells[:, 1] + nc[1] * cells[:, 2]), -1)
    acc = {"workload": cwl.name, "particles": cwl.n, "steps": k,
           "note": "relative L2 of the state and of its increments since step 0 (disp, dvol), and the largest "
                   "per-particle error over the field's RMS (max_rms); the FP32 offset resolves 3e-8 cells, "
                   "so disp errors below ~1e-7 cells x steps^-2 are that resolution, not arithmetic"}
    for pname, prec in (("fp32_mixed", W.FP32_MIXED), ("fp64_plain", W.FP64_PLAIN)):
        with mpm.Simulation(cwl, precision=prec, stream=sptr) as g:
            s0, _ = g.read(("pos", "vol"))
            g.step(k)
            snap, gst = g.read(("pos", "vel", "stress", "vol", "cell"))
        live = (snap["cell"] >= 0) & (ref_cell >= 0)
        disp_g, disp_r = (snap["pos"] - s0["pos"])[live], (st.x[:, :d] - cwl.pos)[live]
        acc[pname] = {
            "disp": _rel_l2(disp_g, disp_r), "disp_max_rms": _max_over_rms(disp_g, disp_r),
            "vel": _rel_l2(snap["vel"][live], st.v[live, :d]),
            "vel_max_rms": _max_over_rms(snap["vel"][live], st.v[live, :d]),
            "stress": _rel_l2(snap["stress"][live], st.sig[live]),
            "stress_max_rms": _max_over_rms(snap["stress"][live], st.sig[live]),
            "dvol": _rel_l2((snap["vol"] - s0["vol"])[live], (st.vol - cwl.vol)[live]),
            "cells_differing": int((snap["cell"] != ref_cell).sum()),
            "status": mpm.STATUS_NAMES.get(gst, gst),
        }
    del o
    rate_all, cores, ks = cpu_oracle_all_cores(name, budget_s, max_steps)
    what = (f"the full {cwl.n}-particle workload" if name == wl_name else
            f"{cwl.name} ({cwl.n} particles, sample of {wl_name})")
    cpu = {"value": rate_all, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": f"FP64 oracle, one replica per core, first {min(ks)}-{max(ks)} steps of {what}; "
                     f"all replicas' particle-steps / slowest replica's time",
           "single_thread": {"value": rate, "cores": 1, "steps": k, "seconds": round(dt, 2)}}
    return cpu, acc


def run_reference(args):
    """The oracle as it stands, one thread, on the bounded sample of the
    workload; every step is one oracle step of the sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    name = CPU_SAMPLE[args.workload]
    wl = make_workload(name)
    o = oracle.from_workload(wl)
    t_w0 = time.perf_counter()
    for _ in range(args.warmup):
        o.step(1)
    t_step = (time.perf_counter() - t_w0) / max(args.warmup, 1)
    k = args.steps
    cap = max(1, int(math.ceil(120.0 / max(t_step, 1e-6))))
    k_timed = min(k, cap)
    t0 = time.perf_counter()
    for _ in range(k_timed):
        o.step(1)
    dt = time.perf_counter() - t0
    value = wl.n * k_timed / dt
    sample = (f"steps {args.warmup + 1}..{args.warmup + k_timed} of {wl.name} ({wl.n} particles"
              + ("" if name == args.workload else f", the bounded sample of {args.workload}")
              + "), FP64 oracle, one thread" + ("" if k_timed == k else f" (capped at {k_timed} of {k} steps)"))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": k_timed, "warmup": args.warmup, "ms_per_step": 1e3 * dt / k_timed,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": make_workload_name(args.workload), "sample": wl.name,
                                            "particles": wl.n},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


WORKLOAD_NAMES = {"slope": "slope_3d_800x200x200"}   # built without its 63.9M particles


def make_workload_name(name):
    return WORKLOAD_NAMES[name] if name in WORKLOAD_NAMES else make_workload(name).name


def run_batched(args, flush, stream):
    """256 independent 2D granular columns (5k-60k particles each) advanced by
    batched steps (one launch per phase over all of them), against stepping
    the same meshes one after another."""
    import torch
    from paper_1909_13380_gb300 import mpm
    wls = W.columns2d_batch(count=args.batch_count)
    ntot = sum(w.n for w in wls)
    sims = [mpm.Simulation(w, stream=C.c_void_p(stream.cuda_stream)) for w in wls]
    b = mpm.mpm_batch_create(stream.cuda_stream, max_slots=len(sims))
    k = max(1, min(args.steps, 20))
    try:
        for s_ in sims:
            mpm.mpm_batch_admit(b, s_.h)
        with torch.cuda.stream(stream):
            # into the collapse first, as the headline: the timed steps are
            # advance + warmup + 1 .. advance + warmup + k
            mpm.mpm_batch_step(b, args.advance + args.warmup)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
            for i in range(k):
                ev[i][0].record(stream)
                mpm.mpm_batch_step(b, 1)
                ev[i][1].record(stream)
                flush.zero_()
        stream.synchronize()
        ms = [a.elapsed_time(c) for a, c in ev]
        status = mpm.mpm_batch_poll(b, len(sims))
        kernels = mpm.mpm_batch_step_kernels(b)
        for i in range(len(sims)):
            mpm.mpm_batch_evict(b, i)
        # the same meshes stepped one at a time (each mesh its own launches)
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s_ in sims:
                s_.step(1)
            e1.record(stream)
        stream.synchronize()
        ms_seq = e0.elapsed_time(e1)
    finally:
        mpm.mpm_batch_destroy(b)
        for s_ in sims:
            s_.close()
    ms_step = float(np.median(ms))
    return {"workload": f"{len(wls)} independent 2D granular columns, 5k-60k particles each (log-uniform)",
            "particles": int(ntot), "value": ntot / (ms_step * 1e-3), "unit": METRIC,
            "ms_per_batched_step": ms_step, "steps": k,
            "timed_steps": f"{args.advance + args.warmup + 1}..{args.advance + args.warmup + k}",
            "one_at_a_time": {"value": ntot / (ms_seq * 1e-3), "ms_per_step_of_all": ms_seq},
            "batching_speedup": ms_seq / ms_step,
            "failed": int(sum(1 for x in status if x != mpm.MPM_OK)),
            "gpu_launches_per_batched_step": kernels}


def serve_session(reqs, chunk):
    """One session of `reqs` with continuous batching (FP32 mixed) and one at
    a time in plain FP64.  Request inputs are built on a background thread a
    few requests ahead of their arrival and dropped once on the device."""
    from paper_1909_13380_gb300 import serve
    out = {}
    for name, kw in (("fp32_continuous_batching", dict(batched=True)),
                     ("fp64_one_at_a_time", dict(precision=W.FP64_PLAIN, batched=False))):
        eng = serve.GpuEngine(**kw)
        stream = serve.RequestStream(reqs, lambda r: r.workload(), ahead=16)
        try:
            done, lat, total = serve.Server(eng, chunk=chunk).run(reqs, stream)
        finally:
            stream.close()
            eng.shutdown()
        rep = serve.report(done, lat, total)
        rep["h2d_bytes"], rep["d2h_bytes"] = eng.h2d, eng.d2h
        out[name] = rep
    return out


def run_serving(args):
    """Poisson stream of mixed 2D/3D column and slope requests served with
    continuous batching (FP32 mixed) and one at a time in plain FP64, at
    20 requests/s; with --serve-rates, the same requests at other rates too
    (arrival times scaled)."""
    reqs = W.serving_requests(count=args.serve_requests, step_scale=args.serve_step_scale)
    out = {"requests": len(reqs), "arrival_rate_per_s": 20.0,
           "sample": f"{len(reqs)} requests, 1e4-4e6 particles (log-uniform), 1000-20000 steps (log-uniform) "
                     f"x {args.serve_step_scale:g}, kinds {'/'.join(W.REQUEST_KINDS)}"}
    out.update(serve_session(reqs, args.serve_chunk))
    rates = [float(x) for x in args.serve_rates.split(",") if x] if args.serve_rates else []
    if rates:
        sweep = []
        for rate in rates:
            scaled = [dataclasses.replace(r, arrival=r.arrival * 20.0 / rate) for r in reqs]
            res = serve_session(scaled, args.serve_chunk)
            sweep.append({"arrival_rate_per_s": rate, **{
                k: {m: res[k][m] for m in ("session_s", "utilisation", "step_ms", "e2e_s", "queue_s")}
                for k in res}})
        out["rate_sweep"] = sweep
    return out




def timed_steps(sim, k, stream, flush):
    """k steps of sim, each bracketed by CUDA events on the library's stream,
    the L2 flushed between them; returns the per-step milliseconds."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    with torch.cuda.stream(stream):
        for i in range(k):
            ev[i][0].record(stream)
            sim.step(1)
            ev[i][1].record(stream)
            flush.zero_()
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def advance(sim, steps, stream, chunk=200):
    """Untimed steps, enqueued in chunks."""
    import torch
    with torch.cuda.stream(stream):
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            sim.step(k)
            done += k
    stream.synchronize()


def pinned_like(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    out = t.numpy()
    out[...] = a
    return out, t


def run_mapped(args, stream, sptr, flush):
    """The step on a mapped (isoparametric) mesh: a granular column on
    terrain-following cells (983,040 particles, 160 x 48 x 64 cells), FP32
    mixed and plain FP64, timed like the headline, beside the Cartesian steps
    of the same particle count; and the paper's locate case, 150,000
    particles placed in a mesh of 23,000 mapped cells (the add call: upload,
    initialisation and the neighbourhood walk of every particle, wall clock,
    best of 3)."""
    from paper_1909_13380_gb300 import mpm

    h = 0.005
    wl = W.terrain_column(3, ncells=(160, 48, 64), col_cells=(80, 48, 32), h=h)
    flat = dataclasses.replace(wl, node_xyz=None, pos=W.gauss_fill(W.box_cells((0, 0, 0), (80, 48, 32)), h,
                                                                   (0.0, 0.0, 0.0), 3),
                               vol=np.full(wl.n, h ** 3 / 8.0), name="granular_column_3d_160x48x64_flat")
    k = max(1, min(args.steps, 20))
    out = {"workload": wl.name, "particles": wl.n, "scheme": "USL", "steps": k}
    f32 = dict(precision=W.FP32_MIXED)
    for key, w in (("fp32_ms", dataclasses.replace(wl, **f32)), ("cartesian_fp32_ms", dataclasses.replace(flat, **f32)),
                   ("fp64_ms", wl), ("cartesian_fp64_ms", flat)):
        sim = mpm.Simulation(w, stream=sptr)
        advance(sim, 20, stream)
        timed_steps(sim, args.warmup, stream, flush)
        out[key] = sum(timed_steps(sim, k, stream, flush)) / k
        st = sim.sync()
        sim.close()
        if st != mpm.MPM_OK:
            raise SystemExit(f"mapped leg: {mpm.STATUS_NAMES.get(st, st)}")
    loc = W.terrain_column(3, ncells=(40, 24, 24), col_cells=(40, 24, 20), h=h)
    best = None
    for _ in range(3):
        empty = dataclasses.replace(loc, pos=loc.pos[:0], vel=loc.vel[:0], vol=loc.vol[:0])
        with mpm.Simulation(empty, stream=sptr) as sim:
            stream.synchronize()
            t0 = time.perf_counter()
            mpm.mpm_add_particles(sim.h, loc.pos, loc.vel, loc.vol, sim.mat)
            t = time.perf_counter() - t0
        best = t if best is None else min(best, t)
    out.update({"locate_particles": loc.n, "locate_cells": 40 * 24 * 24, "locate_ms": 1e3 * best})
    return out


def short_floats(obj, digits=6):
    """The JSON line with every float to `digits` significant digits."""
    if isinstance(obj, float):
        return float(f"{obj:.{digits}g}")
    if isinstance(obj, dict):
        return {k: short_floats(v, digits) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [short_floats(v, digits) for v in obj]
    return obj


def run_gb300(args):
    import torch
    from paper_1909_13380_gb300 import mpm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    wl = make_workload(args.workload)
    stream = torch.cuda.Stream(device=device)
    sptr = C.c_void_p(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    detail = {}

    # ---- device-timed steps -------------------------------------------------
    # The run is first brought to its middle (A untimed steps), then W warm-up
    # steps, then the K timed steps of the step graph as a user gets it
    # (kernels chained by programmatic dependent launch).  Per-kernel phase
    # times come from a second pass of K steps whose graph carries event
    # nodes between the kernels (which also serialises them).
    sim = mpm.Simulation(wl, stream=sptr)
    advance(sim, args.advance, stream)
    timed_steps(sim, args.warmup, stream, flush)
    per_step_kernels = mpm.mpm_step_kernels(sim.h)
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    barrier(world)
    step_ms = timed_steps(sim, args.steps, stream, flush)
    barrier(world)
    clocks = sampler.stop()
    t_dev = sum(step_ms) / 1e3
    first = args.advance + args.warmup + 1
    mpm.mpm_set_phase_timing(sim.h, True)
    phases = []
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            sim.step(1)
            phases.append(mpm.mpm_phase_times(sim.h))
            flush.zero_()
    stream.synchronize()
    status = sim.sync()
    if status != mpm.MPM_OK:
        raise SystemExit(f"step failed: {mpm.STATUS_NAMES.get(status, status)}")
    t_max = reduce_max(t_dev, world, device)
    value = world * wl.n * args.steps / t_max
    ph_mean = np.array(phases).mean(axis=0)
    names = ["binning", "p2g", "node", "g2p"] if wl.scheme == W.USL else \
        ["binning", "p2g_mom", "node_v", "g2p_stress", "p2g_force", "node_a", "g2p_advect"]
    ab = algorithmic_bytes(wl.dim, wl.coh is not None)
    peak, peak_kind = load_peak()
    kernels = {"p2g": ph_mean[1], "g2p": ph_mean[3]} if wl.scheme == W.USL else \
        {"p2g": ph_mean[1] + ph_mean[4], "g2p": ph_mean[3] + ph_mean[6]}
    dom = max(kernels, key=kernels.get)
    achieved = ab[dom] * wl.n / (kernels[dom] * 1e-3) / 1e9
    traffic, traffic_src = load_traffic(dom, args.workload, wl.n)
    step_gbs = ab["step"] * wl.n / (t_dev / args.steps) / 1e9
    mpm.mpm_set_phase_timing(sim.h, False)
    sim.close()

    # ---- plain FP64 GPU step on the same workload (from its initial state) --
    fp64 = None
    if not args.no_fp64:
        k64 = max(1, min(args.steps, 10))
        s64 = mpm.Simulation(wl, precision=W.FP64_PLAIN, stream=sptr)
        timed_steps(s64, 1, stream, flush)
        ms64 = sum(timed_steps(s64, k64, stream, flush)) / k64
        s64.close()
        fp64 = {"ms_per_step": ms64, "value": wl.n / (ms64 * 1e-3), "steps": k64,
                "fp32_mixed_speedup": ms64 / (1e3 * t_dev / args.steps)}

    # ---- the other update order (USF when the headline is USL) --------------
    other = None
    if not args.no_usf:
        osch = W.USF if wl.scheme == W.USL else W.USL
        ko = max(1, min(args.steps, 20))
        so = mpm.Simulation(wl, scheme=osch, stream=sptr)
        advance(so, args.advance, stream)
        timed_steps(so, args.warmup, stream, flush)
        mso = sum(timed_steps(so, ko, stream, flush)) / ko
        # per-kernel phases of the same steps, as for the headline
        mpm.mpm_set_phase_timing(so.h, True)
        oph = []
        with torch.cuda.stream(stream):
            for _ in range(ko):
                so.step(1)
                oph.append(mpm.mpm_phase_times(so.h))
                flush.zero_()
        stream.synchronize()
        mpm.mpm_set_phase_timing(so.h, False)
        sto = so.sync()
        onames = ["binning", "p2g", "node", "g2p"] if osch == W.USL else \
            ["binning", "p2g_mom", "node_v", "g2p_stress", "p2g_force", "node_a", "g2p_advect"]
        other = {"scheme": "USF" if osch == W.USF else "USL", "value": wl.n / (mso * 1e-3), "ms_per_step": mso,
                 "steps": ko, "timed_steps": f"{args.advance + args.warmup + 1}..{args.advance + args.warmup + ko}",
                 "phases_ms": dict(zip(onames, [round(float(x), 5) for x in np.array(oph).mean(axis=0)])),
                 "status": mpm.STATUS_NAMES.get(sto, sto), "gpu_launches_per_step": mpm.mpm_step_kernels(so.h)}
        so.close()

    # ---- end to end through the C-ABI with pinned host buffers ---------------
    e2e = None
    if not args.no_e2e:
        fields = ("pos", "vel", "stress")
        pin_in = {k: pinned_like(getattr(wl, k)) for k in ("pos", "vel", "vol") + (("coh",) if wl.coh is not None
                                                                                     else ())}
        wl_pinned = dataclasses.replace(wl, **{k: v[0] for k, v in pin_in.items()})
        pin_out = {k: pinned_like(np.zeros((wl.n, wl.dim if k != "stress" else 6))) for k in fields}
        out = {k: v[0] for k, v in pin_out.items()}
        h2d = sum(v[0].nbytes for v in pin_in.values())
        d2h = sum(a.nbytes for a in out.values())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = mpm.Simulation(wl_pinned, stream=sptr)
        s.step(args.steps)
        snap, st = s.read(fields, out=out)
        s.close()
        t1 = time.perf_counter()
        e2e = {"value": wl.n * args.steps / (t1 - t0), "unit": METRIC,
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "seconds": round(t1 - t0, 4),
               "includes": "create, upload (pinned), K steps, read pos/vel/stress (pinned)"}

    # ---- the mapped (isoparametric) FP64 step (rank 0) ------------------------
    mapped = None
    if rank == 0 and not args.no_mapped:
        mapped = run_mapped(args, stream, sptr, flush)
        detail["mapped"] = mapped

    # ---- batched small meshes and the serving loop (rank 0) -----------------
    batched = serving = None
    if rank == 0 and not args.no_batch:
        batched = run_batched(args, flush, stream)
        detail["batched"] = batched
    if rank == 0 and not args.no_serving:
        serving = run_serving(args)
        detail["serving"] = serving

    # ---- CPU oracle baseline and accuracy (rank 0, N = 1) ---------------------
    cpu = accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, accuracy = cpu_leg(args.workload, args.cpu_budget, args.cpu_steps, sptr)
        detail["accuracy"] = accuracy

    if rank == 0:
        def short_serving(sv):
            if not sv:
                return None
            out = {"requests": sv["requests"], "rate_per_s": sv["arrival_rate_per_s"]}
            for k, nm in (("fp32_continuous_batching", "fp32_batched"), ("fp64_one_at_a_time", "fp64_one_by_one")):
                r = sv[k]
                out[nm] = {"step_ms_p50_p99": [round(r["step_ms"]["p50"], 4), round(r["step_ms"]["p99"], 4)],
                           "e2e_s_p50_p99": [round(r["e2e_s"]["p50"], 4), round(r["e2e_s"]["p99"], 4)],
                           "failed": r["failed"]}
            return out

        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "particles": wl.n, "scheme": "USL" if wl.scheme == W.USL else "USF",
                       "precision": "fp32_mixed", "timed_steps": f"{first}..{first + args.steps - 1}",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": KERNEL_NAMES[dom], "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, **({"traffic_source": traffic_src} if traffic_src else {}),
                         "algorithmic_bytes_per_particle": ab[dom], "ms_per_launch": kernels[dom],
                         "step_achieved": step_gbs, "step_frac": step_gbs / peak,
                         "step_bytes_per_particle": ab["step"],
                         "fp64_plain_ms_per_step": fp64["ms_per_step"] if fp64 else None,
                         "fp32_vs_fp64_plain": fp64["fp32_mixed_speedup"] if fp64 else None},
            "phases_ms": dict(zip(names, [round(float(x), 5) for x in ph_mean])),
            "clocks": clocks, "gpu_launches": per_step_kernels * args.steps,
            "e2e": e2e, "cpu_baseline": cpu,
            "accuracy": None if not accuracy else {
                "sample": accuracy["workload"], "steps": accuracy["steps"],
                **{p: {k: accuracy[p][k] for k in ("disp", "vel", "stress", "dvol", "stress_max_rms",
                                                   "cells_differing")} for p in ("fp32_mixed", "fp64_plain")}},
            "other_scheme": None if not other else {k: other[k] for k in ("scheme", "ms_per_step", "value",
                                                                          "phases_ms")},
            "batched": None if not batched else {k: batched[k] for k in ("particles", "value", "ms_per_batched_step",
                                                                       "batching_speedup")},
            "serving": short_serving(serving),
            "mapped": None if not mapped else {k: mapped[k] for k in ("workload", "fp32_ms", "cartesian_fp32_ms",
                                                                      "fp64_ms", "cartesian_fp64_ms",
                                                                      "locate_particles", "locate_cells",
                                                                      "locate_ms")},
        }
        line = short_floats(line)
        detail.update({"fp64_plain": fp64, "other_scheme": other, "e2e": e2e, "phases_ms_all": phases,
                       "step_ms": step_ms})
        if args.detail_out:
            with open(args.detail_out, "w") as f:
                json.dump(detail, f, indent=1, default=float)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--advance", type=int, default=1000, help="untimed steps before the warm-up")
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", default="slope", choices=sorted(CPU_SAMPLE))
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-usf", action="store_true", help="skip the other update order (USF)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-steps", type=int, default=200, help="most oracle steps of the CPU sample")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256 batched 2D columns")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving session")
    ap.add_argument("--no-mapped", action="store_true", help="skip the FP64 step on a mapped mesh")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-step-scale", type=float, default=1.0 / 50)
    ap.add_argument("--serve-chunk", type=int, default=16)
    ap.add_argument("--serve-rates", default="", help="also serve the requests at these arrival rates, e.g. 2,5,10,20")
    ap.add_argument("--detail-out", default="", help="write the full detail of every leg as JSON here")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
