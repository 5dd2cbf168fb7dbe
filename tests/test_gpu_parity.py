"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the
same seeded inputs (sizes that span several tiles with ragged tails, and the
full 512,000-particle column in the configuration the benchmark times).

Bars: cells and binning bit-exact; FP64 GPU within 1e-9 relative L2 of the
oracle; FP32 mixed within 1e-5 per step from an identical state and 1e-3
after a run (tests/helpers.py).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1909_13380_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected only with -m gpu on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1909_13380_gb300 import mpm  # noqa: E402


def run_gpu(wl, steps, precision=None, scheme=None):
    with mpm.Simulation(wl, precision=precision, scheme=scheme) as sim:
        if steps:
            sim.step(steps)
        snap, st = sim.read()
        return snap, st


def run_oracle(wl, steps, scheme=None):
    o = H.oracle_from_workload(wl, scheme)
    st = o.step(steps) if steps else oracle.OK
    return H.oracle_snapshot(o, wl.dim), st


@pytest.mark.parametrize("precision", [W.FP64_PLAIN, W.FP32_MIXED])
def test_initial_cells_bit_exact(precision):
    wl = H.small_column(precision=precision)
    gpu, st = run_gpu(wl, 0)
    ref, _ = run_oracle(wl, 0)
    assert st == mpm.MPM_OK
    assert np.array_equal(gpu["cell"], ref["cell"])


@pytest.mark.parametrize("precision", [W.FP64_PLAIN, W.FP32_MIXED])
def test_initial_state_matches_the_inputs(precision):
    # the FP32 storage is formed on the device from the FP64 inputs: offsets
    # round to FP32 once, so positions read back lie within the offset's
    # resolution (2^-24 cells) of the inputs; mass and velocity are the
    # inputs rounded to FP32
    wl = H.small_column(precision=precision)
    rng = np.random.default_rng(3)
    wl = dataclasses.replace(wl, vel=rng.normal(0.0, 0.1, wl.vel.shape))
    s0 = rng.normal(0.0, 1e3, (wl.n, 6))
    with mpm.Simulation(wl, stress0=s0) as sim:
        g, st = sim.read()
    assert st == mpm.MPM_OK
    tol = 1e-15 if precision == W.FP64_PLAIN else 2.0 ** -24
    assert np.abs(g["pos"] - wl.pos).max() <= tol * wl.h * 1.01
    f32 = (lambda a: a) if precision == W.FP64_PLAIN else (lambda a: a.astype(np.float32).astype(np.float64))
    assert np.array_equal(g["vel"], f32(wl.vel))
    assert np.array_equal(g["stress"][:, :6], f32(s0))
    assert np.allclose(g["vol"], wl.vol, rtol=1e-7, atol=0.0)
    assert not g["strain"].any() and not g["epsp"].any()


@pytest.mark.parametrize("precision", [W.FP64_PLAIN, W.FP32_MIXED])
def test_add_particles_rejects_points_outside_the_mesh(precision):
    wl = H.small_column(precision=precision)
    with mpm.Simulation(wl) as sim:
        n = mpm.mpm_num_particles(sim.h)
        upper = np.array(wl.ncells[:3], float) * wl.h
        for bad_x in (-1e-6, upper[0], float("nan")):
            pos = wl.pos[:7].copy()
            pos[3, 0] = bad_x
            with pytest.raises(mpm.MPMError) as ei:
                mpm.mpm_add_particles(sim.h, pos, wl.vel[:7], wl.vol[:7], sim.mat)
            assert ei.value.status == mpm.MPM_ERR_ARG
        # the mesh is unchanged and still steps; a valid add then succeeds
        assert mpm.mpm_num_particles(sim.h) == n
        sim.step(2)
        assert sim.sync() == mpm.MPM_OK
        assert mpm.mpm_add_particles(sim.h, wl.pos[:7], wl.vel[:7], wl.vol[:7], sim.mat) == n
        sim.step(1)
        assert sim.sync() == mpm.MPM_OK


def test_fp64_bar_matches_oracle():
    wl = W.elastic_bar()
    start, _ = run_oracle(wl, 0)
    gpu, st = run_gpu(wl, wl.steps)
    ref, rst = run_oracle(wl, wl.steps)
    assert st == mpm.MPM_OK and rst == oracle.OK
    err = H.compare(gpu, ref, start, 2)
    assert max(err.values()) <= H.TOL_RUN_FP64, err
    assert np.array_equal(gpu["cell"], ref["cell"])


@pytest.mark.parametrize("scheme", [W.USF, W.USL])
def test_fp32_bar(scheme):
    wl = W.elastic_bar(precision=W.FP32_MIXED, scheme=scheme)
    start, _ = run_oracle(wl, 0, scheme)
    g1, _ = run_gpu(wl, 1)
    r1, _ = run_oracle(wl, 1, scheme)
    H.check_step(g1, r1, start, wl.h, 2)
    gpu, st = run_gpu(wl, wl.steps)
    ref, _ = run_oracle(wl, wl.steps, scheme)
    assert st == mpm.MPM_OK
    err = H.compare(gpu, ref, start, 2)
    assert H.worst(err, H.RUN_KEYS) <= H.TOL_RUN_FP32, err


@pytest.mark.parametrize("scheme", [W.USL, W.USF])
def test_small_column_fp64(scheme):
    wl = H.small_column(precision=W.FP64_PLAIN, scheme=scheme)
    start, _ = run_oracle(wl, 0, scheme)
    gpu, st = run_gpu(wl, 200)
    ref, _ = run_oracle(wl, 200, scheme)
    assert st == mpm.MPM_OK
    err = H.compare(gpu, ref, start, 3)
    assert max(err.values()) <= H.TOL_RUN_FP64, err
    ndiff, nout = H.cell_mismatch_in_band(gpu, ref, wl.h, 1e-6)
    assert nout == 0


@pytest.mark.parametrize("scheme", [W.USL, W.USF])
def test_small_column_fp32(scheme):
    wl = H.small_column(precision=W.FP32_MIXED, scheme=scheme)
    start, _ = run_oracle(wl, 0, scheme)
    g1, _ = run_gpu(wl, 1)
    r1, _ = run_oracle(wl, 1, scheme)
    H.check_step(g1, r1, start, wl.h, 3)
    gpu, st = run_gpu(wl, 300)
    ref, _ = run_oracle(wl, 300, scheme)
    assert st == mpm.MPM_OK
    err = H.compare(gpu, ref, start, 3)
    assert H.worst(err, H.RUN_KEYS) <= H.TOL_RUN_FP32, err
    assert H.disp_excess(gpu, ref, start, wl.h, 300, 3) <= 1.0
    ndiff, nout = H.cell_mismatch_in_band(gpu, ref, wl.h, 1e-4)
    assert nout == 0


def test_full_column_per_step_parity():
    """512,000 particles, FP32 USL, the benchmark's launch configuration:
    one step from the initial state, then one step from a developed state
    (the GPU's own state after 60 steps), each against the oracle."""
    wl = W.column3d()
    start, _ = run_oracle(wl, 0)
    with mpm.Simulation(wl) as sim:
        sim.step(1)
        g1, st = sim.read()
        assert st == mpm.MPM_OK
        r1, _ = run_oracle(wl, 1)
        H.check_step(g1, r1, start, wl.h, 3)
        sim.step(59)
        s60, st = sim.read()
        assert st == mpm.MPM_OK
        sim.step(1)
        g61, _ = sim.read()
    o = H.oracle_from_gpu(wl, s60)
    assert o.step(1) == oracle.OK
    r61 = H.oracle_snapshot(o, 3)
    H.check_step(g61, r61, s60, wl.h, 3)
    assert H.cell_mismatch_in_band(g61, r61, wl.h, 1e-4)[1] == 0


WIDE_MESH = {"mid": (100, 40, 48), "wide": (120, 48, 48), "wider": (260, 64, 64)}


@pytest.mark.parametrize("mesh", ["small", "mid", "wide", "wider"])
def test_binning_is_the_stable_sort_of_the_keys(mesh):
    # small: 240 tiles (the one-CTA tile scan, one tile per thread); mid:
    # 3000 tiles (one-CTA scan, three 32-tile chunks per warp, the last warp's
    # ragged); wide: 4320 tiles, past the one-CTA scan's 4096 (the look-back
    # scan over five CTAs); wider: 16,640 tiles (look-back over 17 CTAs)
    wl = H.small_column() if mesh == "small" else W.column3d(ncells=WIDE_MESH[mesh], col_cells=(12, 12, 12))
    with mpm.Simulation(wl) as sim:
        sim.step(37)
        key, perm, td = sim.binning()
        snap, _ = sim.read(fields=("cell", "pos"))
    assert np.array_equal(perm, np.argsort(key, kind="stable").astype(np.int32))
    # keys are the tile-major ids of the cells
    nc = wl.ncells
    c = snap["cell"]
    ix, iy, iz = c % nc[0], (c // nc[0]) % nc[1], c // (nc[0] * nc[1])
    nt = [-(-nc[k] // td[k]) for k in range(3)]
    t = ix // td[0] + nt[0] * (iy // td[1] + nt[1] * (iz // td[2]))
    loc = ix % td[0] + td[0] * (iy % td[1] + td[1] * (iz % td[2]))
    expect = t * (td[0] * td[1] * td[2]) + loc
    assert np.array_equal(np.sort(key), np.sort(expect.astype(np.int32)))
    # the oracle's locate of each stored (cell, offset) gives the stored cell
    cells = oracle.locate(oracle.Mesh(dim=3, n=nc, h=wl.h), snap["pos"])
    lin = cells[:, 0] + nc[0] * (cells[:, 1] + nc[1] * cells[:, 2])
    bad = lin != c
    if bad.any():
        frac = snap["pos"][bad] / wl.h
        assert np.abs(frac - np.round(frac)).min(axis=1).max() < 1e-9


@pytest.mark.parametrize("n", [0, 1, 31, 33, 4095, 4096, 4097, 100_003])
@pytest.mark.parametrize("bits", [1, 8, 13, 20, 32])
def test_sort_keys_primitive(n, bits):
    rng = np.random.default_rng(n * 31 + bits)
    hi = (1 << bits) if bits < 32 else (1 << 32)
    keys = rng.integers(0, min(hi, 50) if n % 2 else hi, size=n, dtype=np.uint64).astype(np.uint32)
    dk = torch.from_numpy(keys.view(np.int32)).cuda()
    dp = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    mpm.mpm_sort_keys(dk, dp, n, bits)
    torch.cuda.synchronize()
    got = dp[:n].cpu().numpy()
    assert np.array_equal(got, np.argsort(keys, kind="stable").astype(np.int32))


def test_apex_band_returns_inside_a_step():
    # A cohesive block in hydrostatic tension just past the apex c cot(phi),
    # with a small deviator and tiny strain increments: every trial of the
    # step lies in the apex band, so G2P queues it and the FP64 apex-band
    # kernel completes it.  One step from the same state as the oracle.
    c, phi = 10e3, math.radians(30.0)
    pa = c / math.tan(phi)
    base = H.small_column()
    rng = np.random.default_rng(23)
    n = base.n
    wl = dataclasses.replace(base, name="cohesive_block_at_apex", gravity=(0.0, 0.0, 0.0),
                             face_bc=(W.FREE,) * 6, face_mu=(0.0,) * 6,
                             material=dict(base.material, c=c), vel=rng.normal(0.0, 2e-5, (n, 3)))
    s0 = np.zeros((n, 6))
    s0[:, :3] = pa * (1.0 + 2e-4)
    s0 += rng.normal(0.0, 1e-5 * pa, (n, 6))
    with mpm.Simulation(wl, stress0=s0) as sim:
        g0, _ = sim.read()
        sim.step(1)
        g1, st = sim.read()
    assert st == mpm.MPM_OK
    o = H.oracle_from_gpu(wl, g0)
    assert o.step(1) == oracle.OK
    r1 = H.oracle_snapshot(o, 3)
    err = H.compare(g1, r1, g0, 3)
    assert H.worst(err, H.STATE_KEYS) <= H.TOL_STEP_FP32, err
    # most trials went back to the apex region, so the band was exercised
    # (particles near the free faces, where the tension is unbalanced, strain
    # more and leave it)
    apex = np.array([pa, pa, pa, 0.0, 0.0, 0.0])
    at_apex = np.linalg.norm(r1["stress"] - apex, axis=1) < 2e-3 * pa
    assert at_apex.mean() > 0.4
    assert (g1["epsp"][at_apex] > g0["epsp"][at_apex]).all()


def _trials(rng, n, scale, c):
    out = []
    for i in range(n):
        if i % 4 == 3:   # near the apex c cot(phi)
            pa = c / math.tan(math.radians(30.0))
            s = rng.normal(0, 1e-4 * scale, 6)
            s[:3] += pa + rng.normal(0, 1e-4 * scale)
        else:
            s = rng.normal(0, scale, 6)
            s[:3] += rng.normal(-scale, scale)
        out.append(s)
    return np.array(out)


@pytest.mark.parametrize("c", [0.0, 10e3])
def test_material_update_against_oracle(c):
    rng = np.random.default_rng(17)
    n = 4000
    sig = _trials(rng, n, 3e4, c)
    de = rng.normal(0, 2e-4, (n, 6))
    mat_o = oracle.Material(model=oracle.MOHR_COULOMB, E=10e6, nu=0.3, rho=1800.0, phi=math.radians(30), c=c,
                            psi=0.0)
    mat_g = mpm.make_material(model=mpm.MPM_MOHR_COULOMB, E=10e6, nu=0.3, rho=1800.0, phi=math.radians(30),
                              c=c, psi=0.0)
    ref = np.array([oracle.stress_update(mat_o, c, sig[i], de[i])[0] for i in range(n)])
    out64, _ = mpm.mpm_material_update(mat_g, mpm.MPM_FP64_PLAIN, sig, de)
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1.0
    assert np.all(np.abs(out64 - ref) <= 1e-9 * scale)
    # FP32 inputs are rounded first: compare with the oracle on the rounded inputs
    sig32 = sig.astype(np.float32).astype(np.float64)
    de32 = de.astype(np.float32).astype(np.float64)
    ref32 = np.array([oracle.stress_update(mat_o, c, sig32[i], de32[i])[0] for i in range(n)])
    out32, _ = mpm.mpm_material_update(mat_g, mpm.MPM_FP32_MIXED, sig, de)
    assert H.rel_l2(out32, ref32) <= H.TOL_STEP_FP32
    assert np.all(np.abs(out32 - ref32) <= 2e-4 * scale)


@pytest.mark.parametrize("precision", [W.FP64_PLAIN, W.FP32_MIXED])
def test_particle_leaving_the_mesh(precision):
    pos = np.array([[0.05, 0.05], [0.0995, 0.05], [0.05, 0.02]])
    vel = np.array([[0.0, 0.0], [200.0, 0.0], [0.0, 0.0]])
    wl = W.Workload(name="leave", dim=2, ncells=(10, 10, 1), h=0.01, origin=(0, 0, 0), face_bc=(0,) * 6,
                    face_mu=(0,) * 6, gravity=(0, 0, 0), dt=1e-5, scheme=W.USL, precision=precision,
                    material=dict(model=0, E=1e3, nu=0.2, rho=1000.0, phi=0, c=0, psi=0), pos=pos, vel=vel,
                    vol=np.full(3, 2.5e-5))
    with mpm.Simulation(wl) as sim:
        sim.step(5)
        assert sim.sync() == mpm.MPM_ERR_LEFT_MESH
        snap, st = sim.read()
    assert st == mpm.MPM_ERR_LEFT_MESH
    assert snap["cell"][1] == -1 and snap["cell"][0] >= 0 and snap["cell"][2] >= 0
    assert np.all(np.isfinite(snap["pos"][[0, 2]]))


@pytest.mark.parametrize("precision", [W.FP64_PLAIN, W.FP32_MIXED])
def test_empty_and_single_particle(precision):
    wl = W.elastic_bar(precision=precision)
    empty = W.Workload(**{**wl.__dict__, "pos": wl.pos[:0], "vel": wl.vel[:0], "vol": wl.vol[:0]})
    with mpm.Simulation(empty) as sim:
        sim.step(3)
        assert sim.sync() == mpm.MPM_OK
        cons, _ = sim.conservation()
        assert cons["alive"] == 0
    # one particle in free fall, crossing cells: v = n g dt, x = x0 + g dt^2 n(n+1)/2
    g = (0.7, 0.4, -9.81)
    one = W.Workload(name="one", dim=3, ncells=(40, 40, 40), h=0.01, origin=(0, 0, 0), face_bc=(0,) * 6,
                     face_mu=(0,) * 6, gravity=g, dt=1e-3, scheme=W.USL, precision=precision,
                     material=dict(model=0, E=10.0, nu=0.2, rho=1000.0, phi=0, c=0, psi=0),
                     pos=np.array([[0.2031, 0.3507, 0.3313]]), vel=np.zeros((1, 3)), vol=np.array([1e-6]))
    with mpm.Simulation(one) as sim:
        sim.step(100)
        snap, st = sim.read()
    assert st == mpm.MPM_OK
    tol = 1e-12 if precision == W.FP64_PLAIN else 1e-5
    assert np.allclose(snap["vel"][0], 100 * np.array(g) * 1e-3, rtol=tol, atol=tol)
    expect = one.pos[0] + np.array(g) * 1e-6 * 100 * 101 / 2
    assert np.allclose(snap["pos"][0], expect, rtol=0, atol=tol * 0.5)


def test_fp32_step_is_deterministic():
    wl = H.small_column()
    a, _ = run_gpu(wl, 120)
    b, _ = run_gpu(wl, 120)
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


@pytest.mark.parametrize("precision", [W.FP64_PLAIN, W.FP32_MIXED])
def test_conservation_sums(precision):
    wl = H.small_column(precision=precision)
    with mpm.Simulation(wl) as sim:
        sim.step(50)
        cons, st = sim.conservation()
        snap, _ = sim.read()
    o = H.oracle_from_gpu(wl, snap)
    if precision == W.FP32_MIXED:
        o.state.m[:] = (wl.material["rho"] * wl.vol).astype(np.float32)
    ref = o.conservation()
    assert cons["alive"] == ref["alive"] == wl.n
    assert cons["mass"] == pytest.approx(ref["mass"], rel=1e-12)
    assert np.allclose(cons["momentum"], ref["momentum"], rtol=1e-9, atol=1e-12 * ref["mass"])
    assert cons["ke"] == pytest.approx(ref["ke"], rel=1e-9)
    # strain energy 1/2 V sig:eps and total volume: the FP32 sums form V with
    # the FP32 reciprocal of rho, the read-back with rho itself (6e-8 apart)
    rel_v = 1e-12 if precision == W.FP64_PLAIN else 1e-6
    assert ref["se"] > 0 and cons["se"] == pytest.approx(ref["se"], rel=rel_v)
    alive = o.state.alive == 1
    assert cons["volume"] == pytest.approx(o.state.vol[alive].sum(), rel=rel_v)
    # mass is carried exactly by the particles
    assert cons["mass"] == pytest.approx((wl.material["rho"] * wl.vol).sum(), rel=1e-6)


def test_binning_with_mass_tile_crossing():
    """1,600 particles cross a tile boundary in one step (more arrivals than
    the shared-memory bucket holds): the incremental binning still equals the
    stable sort of the keys, step after step, and P2G conserves the mass."""
    h = 1.0
    cells = W.box_cells((6, 0), (8, 8))
    pos = np.repeat((cells + 0.5) * h, 200, axis=0)
    rng = np.random.default_rng(3)
    pos += rng.uniform(-0.45, 0.45, pos.shape) * h
    vel = np.tile([0.9, 0.0], (pos.shape[0], 1))
    wl = W.Workload(name="crossing", dim=2, ncells=(32, 8, 1), h=h, origin=(0, 0, 0), face_bc=(0,) * 6,
                    face_mu=(0,) * 6, gravity=(0, 0, 0), dt=1.0, scheme=W.USL, precision=W.FP32_MIXED,
                    material=dict(model=0, E=1e-6, nu=0.2, rho=1.0, phi=0, c=0, psi=0), pos=pos, vel=vel,
                    vol=np.full(pos.shape[0], 1.0 / 200))
    with mpm.Simulation(wl) as sim:
        for step in range(4):
            key, perm, td = sim.binning()
            assert np.array_equal(perm, np.argsort(key, kind="stable").astype(np.int32)), step
            sim.step(1)
            assert sim.sync() == mpm.MPM_OK
            cons, _ = sim.conservation()
            assert cons["alive"] == wl.n
            assert cons["mass"] == pytest.approx(wl.n * np.float32(1.0 / 200), rel=1e-6)
        snap, _ = sim.read(fields=("pos",))
    # everything moved about 4 x 0.9 cells to the right
    assert abs(np.mean(snap["pos"][:, 0] - pos[:, 0]) - 3.6) < 0.05


def _degenerate_trials(rng, n, scale):
    """Stress states with repeated or nearly repeated principal values in a
    random frame: axisymmetric (the lateral pair equal, as in a column at
    rest), the other pair equal, near-hydrostatic, and exactly diagonal."""
    out = []
    for i in range(n):
        k = i % 5
        if k == 0:
            lam = np.array([-1.0, -1.0, -2.5])
        elif k == 1:
            lam = np.array([-1.0, -1.0 - rng.uniform(0, 1e-5), -3.0])
        elif k == 2:
            lam = np.array([-0.5, -3.0 + rng.uniform(0, 1e-5), -3.0])
        elif k == 3:
            lam = -2.0 + rng.normal(0, 1e-6, 3)
        else:
            lam = rng.normal(-1.0, 1.0, 3)
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if k == 4:
            q = np.eye(3)
        S = (q * lam) @ q.T * scale
        out.append([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[1, 2], S[0, 2]])
    return np.array(out)


@pytest.mark.parametrize("c", [0.0, 10e3])
def test_material_update_degenerate_spectra(c):
    """The FP32 return uses a closed-form eigen-decomposition with deflation;
    repeated and nearly repeated principal stresses must come out as
    accurately as well-separated ones."""
    rng = np.random.default_rng(23)
    n = 4000
    sig = _degenerate_trials(rng, n, 3e4)
    de = rng.normal(0, 2e-4, (n, 6))
    de[::3] = 0.0   # returns of the trial state itself
    mat_o = oracle.Material(model=oracle.MOHR_COULOMB, E=10e6, nu=0.3, rho=1800.0, phi=math.radians(30), c=c,
                            psi=0.0)
    mat_g = mpm.make_material(model=mpm.MPM_MOHR_COULOMB, E=10e6, nu=0.3, rho=1800.0, phi=math.radians(30),
                              c=c, psi=0.0)
    sig32 = sig.astype(np.float32).astype(np.float64)
    de32 = de.astype(np.float32).astype(np.float64)
    ref32 = np.array([oracle.stress_update(mat_o, c, sig32[i], de32[i])[0] for i in range(n)])
    out32, _ = mpm.mpm_material_update(mat_g, mpm.MPM_FP32_MIXED, sig, de)
    scale = np.abs(ref32).max(axis=1, keepdims=True) + 1.0
    assert H.rel_l2(out32, ref32) <= H.TOL_STEP_FP32
    assert np.all(np.abs(out32 - ref32) <= 2e-4 * scale)


@pytest.mark.parametrize("kind", ["column2d", "slope2d", "slope3d"])
@pytest.mark.parametrize("scheme", [W.USL, W.USF])
def test_request_kinds_fp32(kind, scheme):
    """The other workload kinds the serving loop runs -- 2D Mohr-Coulomb
    column with base friction, 2D and 3D slopes with per-particle cohesion and
    a fixed base -- against the oracle: one step, then a run."""
    wl = W.request_workload(kind, 6e3 if kind != "slope3d" else 1.2e4, seed=W.SEED_BASE + 61, steps=120)
    wl.scheme = scheme
    d = wl.dim
    start, _ = run_oracle(wl, 0, scheme)
    g1, _ = run_gpu(wl, 1)
    r1, _ = run_oracle(wl, 1, scheme)
    H.check_step(g1, r1, start, wl.h, d)
    gpu, st = run_gpu(wl, wl.steps)
    ref, _ = run_oracle(wl, wl.steps, scheme)
    assert st == mpm.MPM_OK
    err = H.compare(gpu, ref, start, d)
    assert H.worst(err, H.RUN_KEYS) <= H.TOL_RUN_FP32, err
    assert H.disp_excess(gpu, ref, start, wl.h, wl.steps, d) <= 1.0
    ndiff, nout = H.cell_mismatch_in_band(gpu, ref, wl.h, 1e-4)
    assert nout == 0


def _fused_vs_full(wl, steps):
    """The same run twice: plain steps, and steps each followed by a scratch
    binning (mpm_read_binning), which must leave the trajectory alone.  It
    also advances the step index, so with the fused USL step (G2P summing the
    next step's P2G of the particles that stay in their tile, a residual P2G
    adding arrivals) every tile's next P2G is recomputed in full from the
    stored state: the comparison is then fused against full sums."""
    with mpm.Simulation(wl) as a, mpm.Simulation(wl) as b:
        for _ in range(steps):
            a.step(1)
            a.binning()
            b.step(1)
        ra, sa = a.read()
        rb, sb = b.read()
    assert sa == sb == mpm.MPM_OK
    return ra, rb


def test_fused_p2g_equals_the_full_p2g_while_no_particle_changes_tile():
    # the first steps of the column from rest: nothing crosses a cell face,
    # so (with the fused step) the fused sums are the plain P2G's, bit for bit
    ra, rb = _fused_vs_full(H.small_column(), 30)
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k


def test_fused_p2g_with_arrivals():
    # every particle crosses into the next tile within four steps: the
    # arrivals' sums go to their own slots, so only the summation order of
    # the nodes differs from the full P2G
    h = 1.0
    cells = W.box_cells((6, 1), (8, 7))
    pos = np.repeat((cells + 0.5) * h, 50, axis=0)
    rng = np.random.default_rng(4)
    pos += rng.uniform(-0.45, 0.45, pos.shape) * h
    vel = np.stack([np.full(pos.shape[0], 0.6), rng.uniform(-0.02, 0.02, pos.shape[0])], axis=1)
    wl = W.Workload(name="crossing_fused", dim=2, ncells=(32, 8, 1), h=h, origin=(0, 0, 0), face_bc=(0,) * 6,
                    face_mu=(0,) * 6, gravity=(0, 0, 0), dt=1.0, scheme=W.USL, precision=W.FP32_MIXED,
                    material=dict(model=0, E=1e-4, nu=0.2, rho=1.0, phi=0, c=0, psi=0), pos=pos, vel=vel,
                    vol=np.full(pos.shape[0], 1.0 / 50))
    ra, rb = _fused_vs_full(wl, 6)
    assert np.array_equal(ra["cell"], rb["cell"])
    for k in ("pos", "vel", "stress", "vol"):
        assert H.rel_l2(ra[k], rb[k]) <= 1e-6, k
    assert abs(np.mean(ra["pos"][:, 0] - pos[:, 0]) - 3.6) < 0.05   # they did move on
