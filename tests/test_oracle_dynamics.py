"""Pins of the oracle's explicit step (CODE OVERVIEW: explicit USF and USL;
INTRODUCTION: nodal values reset each step, particles carry the state;
ISOPARAMETRIC MESH: velocity and frictional conditions at the nodes).

  * a single particle in free fall follows v_n = n g dt and
    x_n = x0 + g dt^2 n (n + 1) / 2 exactly (both schemes, crossing cells);
  * with free faces and no gravity total momentum is conserved; with gravity
    it grows by dt g M per step (sum of grad N = 0 cancels internal forces);
  * the fixed-free elastic bar (64 x 4 quads) matches the closed-form first
    mode: period, tip amplitude and centre-of-mass velocity, with bounded
    energy drift (tests/golden/bar_first_mode.json);
  * a stiff elastic block under inclined gravity on a Coulomb base slides
    with a = g (sin theta - mu cos theta); with mu > tan theta it sticks.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1909_13380_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bar_first_mode.json")


@pytest.mark.parametrize("scheme", [oracle.USF, oracle.USL])
@pytest.mark.parametrize("dim", [2, 3])
def test_single_particle_free_fall(scheme, dim):
    g = (0.7, -9.81, 0.0) if dim == 2 else (0.7, 0.4, -9.81)
    h, dt = 0.01, 1e-3
    mesh = oracle.Mesh(dim=dim, n=(40, 40, 40)[:dim] + (1,) * (3 - dim), h=h, g=g, dt=dt, scheme=scheme)
    x0 = np.array([0.2031, 0.3507, 0.3313][:dim])
    st = oracle.State.create(x0[None, :], np.zeros((1, dim)), [1e-6], rho=1000.0)
    # a soft material keeps dt = 1e-3 below the elastic wave limit h / c
    o = oracle.Oracle(mesh, oracle.Material(E=10.0, nu=0.2), st)
    cells0 = o.cells()[0].copy()
    n = 100
    assert o.step(n) == oracle.OK
    gv = np.array(g[:dim])
    assert np.allclose(st.v[0, :dim], n * gv * dt, rtol=1e-12, atol=1e-14)
    expect = x0 + gv * dt * dt * n * (n + 1) / 2.0
    assert np.allclose(st.x[0, :dim], expect, rtol=1e-12, atol=1e-14)
    assert not np.array_equal(o.cells()[0], cells0)   # it did cross cells


@pytest.mark.parametrize("scheme", [oracle.USF, oracle.USL])
@pytest.mark.parametrize("dim", [2, 3])
def test_momentum_conservation(scheme, dim):
    ncells = (10, 9, 8)[:dim] + (1,) * (3 - dim)
    h = 0.1
    pos, vel, sig, vol = W.random_particles(ncells, h, 400, seed=31 + dim, dim=dim, margin=2,
                                            vel_scale=0.5, sig_scale=1e4)
    mesh = oracle.Mesh(dim=dim, n=ncells, h=h, dt=1e-5, scheme=scheme)
    st = oracle.State.create(pos, vel, vol, rho=1000.0, sig0=sig)
    o = oracle.Oracle(mesh, oracle.Material(E=1e7, nu=0.25), st)
    p0 = o.conservation()["momentum"]
    scale = np.sum(st.m[:, None] * np.abs(st.v))
    assert o.step(20) == oracle.OK
    p1 = o.conservation()["momentum"]
    assert np.all(np.abs(p1 - p0) <= 1e-12 * scale)
    # with gravity the momentum grows by dt g M per step
    g = np.array([0.3, -9.81, 1.1])
    g[dim:] = 0.0
    o.mesh.g = tuple(g)
    M = st.m.sum()
    assert o.step(10) == oracle.OK
    p2 = o.conservation()["momentum"]
    assert np.allclose(p2 - p1, 10 * 1e-5 * g * M, rtol=1e-9, atol=1e-12 * scale)


@pytest.mark.slow
def test_elastic_bar_first_mode():
    ref = json.load(open(GOLDEN))
    wl = W.elastic_bar()
    mesh = oracle.Mesh(dim=2, n=wl.ncells, h=wl.h, face_bc=wl.face_bc, dt=wl.dt, scheme=wl.scheme)
    st = oracle.State.create(wl.pos, wl.vel, wl.vol, wl.material["rho"])
    o = oracle.Oracle(mesh, oracle.Material(**wl.material), st)
    c0 = o.conservation()
    assert c0["mass"] == pytest.approx(ref["mass_per_unit_thickness"], rel=1e-14)
    assert c0["ke"] == pytest.approx(ref["kinetic_energy_0_per_unit_thickness"], rel=1e-12)
    x0 = st.x.copy()
    tip = st.x[:, 0] > wl.meta["L"] - wl.h / 2
    nsteps = int(math.ceil(2.05 * ref["period"] / wl.dt))
    vcm, energy, utip = [], [], []
    for s in range(nsteps):
        assert o.step(1) == oracle.OK
        c = o.conservation()
        vcm.append(c["momentum"][0] / c["mass"])
        energy.append(c["ke"] + c["se"])
        utip.append(np.mean(st.x[tip, 0] - x0[tip, 0]))
    vcm, energy, utip = map(np.array, (vcm, energy, utip))
    t = (np.arange(nsteps) + 1) * wl.dt
    w = ref["omega"]
    # centre-of-mass velocity (2 v0 / pi) cos(w t) at the workload's 2000 steps
    assert abs(vcm[1999] - ref["vcm_amplitude"] * math.cos(w * t[1999])) <= 1e-3 * ref["vcm_amplitude"]
    # period from the zero crossings of the centre-of-mass velocity
    zc = np.nonzero(np.diff(np.sign(vcm)))[0]
    tz = t[zc] - vcm[zc] * (t[zc + 1] - t[zc]) / (vcm[zc + 1] - vcm[zc])
    assert len(tz) >= 4
    assert 2 * np.mean(np.diff(tz)) == pytest.approx(ref["period"], rel=1e-3)
    assert utip.max() == pytest.approx(ref["tip_amplitude"], rel=5e-3)
    assert (energy.max() - energy.min()) / energy[0] < 5e-3


@pytest.mark.slow
@pytest.mark.parametrize("scheme", [oracle.USF, oracle.USL])
def test_block_on_frictional_base(scheme):
    th, g, h = math.radians(30.0), 9.81, 0.05
    pos = W.gauss_fill(W.box_cells((2, 0), (10, 4)), h, (0.0, 0.0), 2)
    res = {}
    for mu in (0.2, 0.8):
        mesh = oracle.Mesh(dim=2, n=(40, 8, 1), h=h, face_bc=(0, 0, 3, 0, 0, 0), face_mu=(0, 0, mu, 0, 0, 0),
                           g=(g * math.sin(th), -g * math.cos(th), 0.0), dt=1e-5, scheme=scheme)
        st = oracle.State.create(pos, np.zeros_like(pos), np.full(len(pos), h * h / 4), 1000.0)
        o = oracle.Oracle(mesh, oracle.Material(E=5e7, nu=0.3, rho=1000.0), st)
        M = st.m.sum()
        n = 5000
        vs = []
        for _ in range(n):
            assert o.step(1) == oracle.OK
            vs.append(np.sum(st.m * st.v[:, 0]) / M)
        t = (np.arange(n) + 1) * 1e-5
        res[mu] = (np.polyfit(t[n // 2:], np.array(vs[n // 2:]), 1)[0], vs[-1])
        # the block never sinks into the base
        assert st.x[:, 1].min() > 0.0
    a_slip = g * (math.sin(th) - 0.2 * math.cos(th))
    assert res[0.2][0] == pytest.approx(a_slip, rel=1e-2)
    assert abs(res[0.8][0]) < 0.05 * a_slip
    assert abs(res[0.8][1]) < 0.1 * abs(res[0.2][1])


def test_node_constraints_by_hand():
    mesh = oracle.Mesh(dim=3, n=(4, 4, 4), h=0.1, dt=1e-3,
                       face_bc=(oracle.BC_FIXED, 0, oracle.BC_ROLLER, 0, oracle.BC_FRICTION, 0),
                       face_mu=(0, 0, 0, 0, 0.5, 0))
    v, a, vn = [1.0, 2.0, 3.0], [10.0, 20.0, 30.0], [1.01, 2.02, 3.03]
    out = oracle.constrain_node(mesh, (0, 2, 2), v, a, vn)          # fixed face
    assert all(np.all(x == 0) for x in out)
    out = oracle.constrain_node(mesh, (2, 0, 2), v, a, vn)          # roller on -y
    assert np.array_equal(out[2], [1.01, 0.0, 3.03]) and out[1][1] == 0.0
    # base (-z, outward -z): moving into the wall at 0.2 m/s -> contact
    v0, a0 = np.array([0.1, 0.0, -0.1]), np.array([0.0, 0.0, -100.0])
    vn0 = v0 + a0 * 1e-3                                             # (0.1, 0, -0.2)
    v, a, vn = oracle.constrain_node(mesh, (2, 2, 0), v0, a0, vn0)
    # Coulomb cap mu * 0.2 = 0.1 >= |vt| = 0.1 -> stick
    assert np.allclose(vn, 0.0) and np.allclose(a, (vn - v0) / 1e-3)
    vn0 = np.array([0.3, 0.0, -0.2])
    v, a, vn = oracle.constrain_node(mesh, (2, 2, 0), v0, a0, vn0)
    assert np.allclose(vn, [0.2, 0.0, 0.0]) and np.allclose(a, (vn - v0) / 1e-3)
    # moving away from the base: untouched
    vn0 = np.array([0.3, 0.0, 0.2])
    v, a, vn = oracle.constrain_node(mesh, (2, 2, 0), v0, a0, vn0)
    assert np.array_equal(vn, vn0) and np.array_equal(a, a0)


# ---------------------------------------------------------------------------
# One explicit step of two particles in one cell, written out by hand from the
# textbook formulas of the two update orders (CODE OVERVIEW: explicit USF and
# USL).  The cell touches the -x face, which is a roller, so the velocity
# condition and the force-stage condition both act.  No oracle routine
# supplies an expected value.
# ---------------------------------------------------------------------------
def _hand_shape(xp, cell, h, origin, d):
    """N_a and dN_a/dx of the linear quad/hex at xp in `cell` (node a: bit k
    of a set = upper node along axis k)."""
    xi = [2.0 * ((xp[k] - origin[k]) / h - cell[k]) - 1.0 for k in range(d)]
    N, G = [], []
    for a in range(1 << d):
        s = [1.0 if (a >> k) & 1 else -1.0 for k in range(d)]
        w = [0.5 * (1.0 + s[k] * xi[k]) for k in range(d)]
        N.append(float(np.prod(w)))
        G.append([s[k] / h * float(np.prod([w[j] for j in range(d) if j != k])) for k in range(d)])
    return np.array(N), np.array(G)


_VOIGT = ((0, 3, 5), (3, 1, 4), (5, 4, 2))   # (xx, yy, zz, xy, yz, xz) -> tensor entry


def _hand_step(scheme, d, P, mesh, E, nu, wrong=None):
    """Expected particle state after one step.  P: dict of x (n,3), v (n,3),
    sig (n,6), eps (n,6), m (n,), vol (n,) with every particle in `cell`.
    `wrong` plants the slips a step-order mistake would make: "usl_strain_v"
    (USL strain from the pre-force v = P/m) or "usf_force_old_sig" (USF
    internal force from the stress at the start of the step)."""
    h, origin, dt, g = mesh.h, mesh.origin, mesh.dt, np.array(mesh.g[:d])
    cell = P["cell"]
    nn = 1 << d
    G_, lam = E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    x, v, sig, eps = P["x"].copy(), P["v"].copy(), P["sig"].copy(), P["eps"].copy()
    m, vol = P["m"].copy(), P["vol"].copy()
    npart = x.shape[0]
    sh = [_hand_shape(x[p], cell, h, origin, d) for p in range(npart)]
    on_roller = [((a & 1) == 0) for a in range(nn)]     # node x index 0: the -x face (roller)

    def mass_momentum():
        mi, Pi = np.zeros(nn), np.zeros((nn, d))
        for p in range(npart):
            N, _ = sh[p]
            for a in range(nn):
                mi[a] += N[a] * m[p]
                Pi[a] += N[a] * m[p] * v[p, :d]
        return mi, Pi

    def force(s6, V):
        f = np.zeros((nn, d))
        for p in range(npart):
            N, Gp = sh[p]
            for a in range(nn):
                for j in range(d):
                    f[a, j] += -V[p] * sum(s6[p, _VOIGT[j][k]] * Gp[a, k] for k in range(d)) + N[a] * m[p] * g[j]
        return f

    def strain_stress(p, vel_nodes):
        N, Gp = sh[p]
        L = np.zeros((3, 3))
        for a in range(nn):
            for j in range(d):
                for k in range(d):
                    L[j, k] += vel_nodes[a, j] * Gp[a, k]
        de = np.array([L[0, 0], L[1, 1], L[2, 2], 0.5 * (L[0, 1] + L[1, 0]), 0.5 * (L[1, 2] + L[2, 1]),
                       0.5 * (L[0, 2] + L[2, 0])]) * dt
        tr = de[0] + de[1] + de[2]
        eps[p] += de
        vol[p] *= 1.0 + tr
        for i in range(3):
            sig[p, i] += lam * tr + 2.0 * G_ * de[i]
        for i in range(3, 6):
            sig[p, i] += 2.0 * G_ * de[i]

    def advect(acc, vnew):
        for p in range(npart):
            N, _ = sh[p]
            v[p, :d] += dt * sum(N[a] * acc[a] for a in range(nn))
            x[p, :d] += dt * sum(N[a] * vnew[a] for a in range(nn))

    mi, Pi = mass_momentum()
    vi = Pi / mi[:, None]
    if scheme == oracle.USL:
        ai = force(sig, vol) / mi[:, None]
        vn = vi + ai * dt
        for a in range(nn):
            if on_roller[a]:
                vi[a, 0] = ai[a, 0] = vn[a, 0] = 0.0
        for p in range(npart):
            strain_stress(p, vi if wrong == "usl_strain_v" else vn)
        advect(ai, vn)
    else:
        for a in range(nn):                  # velocity condition on the pre-force velocity
            if on_roller[a]:
                vi[a, 0] = 0.0
        sig0, vol0 = sig.copy(), vol.copy()
        for p in range(npart):
            strain_stress(p, vi)
        ai = (force(sig0, vol0) if wrong == "usf_force_old_sig" else force(sig, vol)) / mi[:, None]
        vn = vi + ai * dt
        for a in range(nn):
            if on_roller[a]:
                vi[a, 0] = ai[a, 0] = vn[a, 0] = 0.0
        advect(ai, vn)
    return {"x": x, "v": v, "sig": sig, "eps": eps, "vol": vol}


def _two_particle_case(d):
    h, origin = 0.5, (0.1, -0.2, 0.3)
    g = (1.5, -9.81, 0.7)[:d] + (0.0,) * (3 - d)
    mesh = oracle.Mesh(dim=d, n=(3, 3, 3)[:d] + (1,) * (3 - d), h=h, origin=origin,
                       face_bc=(oracle.BC_ROLLER, 0, 0, 0, 0, 0), g=g, dt=1e-2, scheme=oracle.USL)
    cell = (0, 1, 1)[:d] + (0,) * (3 - d)
    frac = np.array([[0.23, 0.61, 0.37], [0.74, 0.18, 0.82]])[:, :d]
    pos = np.array(origin[:d]) + (np.array(cell[:d]) + frac) * h
    vel = np.array([[0.30, -0.12, 0.21], [-0.17, 0.25, -0.08]])[:, :d]
    sig = np.array([[120.0, -80.0, 35.0, 40.0, -22.0, 17.0], [-60.0, 150.0, -45.0, -30.0, 28.0, -11.0]])
    if d == 2:
        sig[:, 4:] = 0.0
    vol = np.array([0.031, 0.027])
    return mesh, cell, pos, vel, sig, vol


@pytest.mark.parametrize("dim", [2, 3])
def test_one_step_order_by_hand(dim):
    E, nu, rho = 1.0e4, 0.25, 900.0
    res = {}
    for scheme in (oracle.USF, oracle.USL):
        mesh, cell, pos, vel, sig, vol = _two_particle_case(dim)
        mesh.scheme = scheme
        st = oracle.State.create(pos, vel, vol, rho, sig0=sig)
        P = {"x": st.x.copy(), "v": st.v.copy(), "sig": st.sig.copy(), "eps": st.eps.copy(), "m": st.m.copy(),
             "vol": st.vol.copy(), "cell": cell}
        expect = _hand_step(scheme, dim, P, mesh, E, nu)
        o = oracle.Oracle(mesh, oracle.Material(E=E, nu=nu, rho=rho), st)
        assert o.step(1) == oracle.OK
        got = {"x": st.x, "v": st.v, "sig": st.sig, "eps": st.eps, "vol": st.vol}
        for k in expect:
            scale = np.abs(expect[k]).max()
            assert np.abs(got[k] - expect[k]).max() <= 1e-13 * scale, (scheme, k)
        # the pin discriminates: the plausible order slips move the result by
        # far more than the tolerance
        slip = "usl_strain_v" if scheme == oracle.USL else "usf_force_old_sig"
        bad = _hand_step(scheme, dim, P, mesh, E, nu, wrong=slip)
        key = "sig" if scheme == oracle.USL else "v"
        assert np.abs(bad[key] - expect[key]).max() > 1e-4 * np.abs(expect[key]).max(), slip
        res[scheme] = got
    # the two orders give different stresses after one step
    d_sig = np.abs(res[oracle.USF]["sig"] - res[oracle.USL]["sig"]).max()
    assert d_sig > 1e-4 * np.abs(res[oracle.USL]["sig"]).max()


# ---------------------------------------------------------------------------
# Plane stress, face tractions and damping: the quasi-static plate with a
# hole of BENCHMARK AND PERFORMANCE (Table 1).
# ---------------------------------------------------------------------------
def test_plane_stress_update_is_the_uniaxial_law():
    # uniaxial stress sigma along x in plane stress: strains sigma/E and
    # -nu sigma/E; the textbook plane-stress matrix E/(1 - nu^2) [[1, nu],
    # [nu, 1]] maps them back to (sigma, 0), with sigma_zz = 0 and the shear
    # 2 G eps_xy
    E, nu = 2.0e7, 0.3
    mat = oracle.Material(model=oracle.PLANE_STRESS_ELASTIC, E=E, nu=nu, rho=1000.0)
    sig0 = np.array([10.0, -4.0, 0.0, 3.0, 0.0, 0.0])
    de = np.array([1e-4, -nu * 1e-4, 0.0, 2e-5, 0.0, 0.0])
    out, depsp = oracle.stress_update(mat, 0.0, sig0, de)
    D = E / (1 - nu * nu)
    expect = sig0 + np.array([D * (de[0] + nu * de[1]), D * (nu * de[0] + de[1]), 0.0,
                              E / (1 + nu) * de[3], 0.0, 0.0])
    assert np.allclose(out, expect, rtol=1e-13, atol=1e-9)
    assert out[1] == pytest.approx(sig0[1], abs=1e-9) and out[2] == 0.0 and depsp == 0.0


@pytest.mark.parametrize("scheme", [oracle.USF, oracle.USL])
def test_face_traction_with_damping_settles_to_the_applied_stress(scheme):
    # a plane-stress bar, roller on -x and -y, traction t on +x, damped to
    # rest: the stress is uniform, sigma_xx = t, sigma_yy = 0, and the strain
    # is the uniaxial plane-stress strain t / E (plane strain would give
    # (1 - nu^2) t / E)
    E, nu, rho, h, t = 1e6, 0.3, 1000.0, 0.1, 50.0
    pos = W.gauss_fill(W.box_cells((0, 0), (12, 2)), h, (0.0, 0.0), 2)
    c = math.sqrt(E / (rho * (1 - nu * nu)))
    trac = [(0.0, 0.0, 0.0)] * 6
    trac[1] = (t, 0.0, 0.0)
    mesh = oracle.Mesh(dim=2, n=(12, 2, 1), h=h, face_bc=(oracle.BC_ROLLER, 0, oracle.BC_ROLLER, 0, 0, 0),
                       dt=0.2 * h / c, scheme=scheme, face_traction=tuple(trac),
                       damping=2.0 * math.pi * c / (2.0 * 1.2))
    st = oracle.State.create(pos, np.zeros_like(pos), np.full(len(pos), h * h / 4), rho)
    o = oracle.Oracle(mesh, oracle.Material(model=oracle.PLANE_STRESS_ELASTIC, E=E, nu=nu, rho=rho), st)
    assert o.step(4000) == oracle.OK
    assert np.allclose(st.sig[:, 0], t, rtol=2e-3)
    assert np.abs(st.sig[:, 1]).max() < 2e-3 * t and not st.sig[:, 2].any()
    assert np.allclose(st.eps[:, 0], t / E, rtol=2e-3)
    assert o.conservation()["ke"] < 1e-12 * rho * 1.2 * 0.2 * c * c


@pytest.mark.slow
def test_plate_with_hole_stress_concentration():
    """BENCHMARK AND PERFORMANCE, Table 1: the quarter strip damped to rest
    under the end traction; the extreme particle stresses at the hole against
    Howland's factors (3.14 for sigma_xx, -1.11 for sigma_yy; the paper's
    USF MPM gave 3.13 and -1.08), and the far field carrying the traction."""
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "plate_with_hole_table1.json")))
    wl = W.plate_with_hole()
    assert abs(wl.n - 40156) <= 5          # the paper's 40,156 material points
    o = oracle.from_workload(wl)
    assert o.step(4000) == oracle.OK
    s0 = wl.meta["sigma0"]
    sx, sy = o.state.sig[:, 0] / s0, o.state.sig[:, 1] / s0
    x = o.state.x[:, 0]
    assert sx.max() == pytest.approx(ref["howland"]["max_sxx"], rel=3e-2)
    assert sy.min() == pytest.approx(ref["howland"]["max_syy"], rel=5e-2)
    assert abs(sx.min()) < 0.25
    assert np.mean(sx[x > 3.5]) == pytest.approx(1.0, abs=2e-3)
