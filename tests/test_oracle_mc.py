"""Pins of the oracle's material update (CODE OVERVIEW: the Material class
turns a strain increment into a stress; Mohr-Coulomb as the granular
material of the column and slope workloads, returned in principal stresses
after de Souza Neto et al. 2008).

Independent pins:
  * the Jacobi eigen-solver against LAPACK (numpy.linalg.eigh);
  * with associated flow (psi = phi) and perfect plasticity the backward-Euler
    return is the closest admissible stress in the complementary-energy norm
    (Simo & Hughes 1998), so every branch -- plane, both edges, apex -- is
    checked against a generic constrained minimiser (scipy SLSQP) over the
    six Mohr-Coulomb planes;
  * with non-associated flow the plastic strain C (sig_tr - sig) must be a
    non-negative combination of the active plastic-potential gradients;
  * a drained triaxial compression driven by strain increments starts with
    slope E (Young's modulus) and saturates at the Rankine passive ratio
    sig_axial / sig_lateral = (1 + sin phi) / (1 - sin phi) (= 3 at 30 deg);
  * hydrostatic tension returns to the apex c cot(phi) (0 when c = 0).
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize, nnls

import oracle

E, NU = 10e6, 0.3
G = E / (2 * (1 + NU))
LAM = E * NU / ((1 + NU) * (1 - 2 * NU))
CMAT = np.array([[1, -NU, -NU], [-NU, 1, -NU], [-NU, -NU, 1]]) / E


def principal(s6):
    S = np.array([[s6[0], s6[3], s6[5]], [s6[3], s6[1], s6[4]], [s6[5], s6[4], s6[2]]])
    return np.sort(np.linalg.eigvalsh(S))[::-1]


def mc_planes(s, phi, c):
    """All six Mohr-Coulomb planes f_ij = (s_i - s_j) + (s_i + s_j) sin phi - 2 c cos phi."""
    out = []
    for i in range(3):
        for j in range(3):
            if i != j:
                out.append((s[i] - s[j]) + (s[i] + s[j]) * math.sin(phi) - 2 * c * math.cos(phi))
    return np.array(out)


def random_trials(rng, n, scale):
    """Random trial stresses: mostly compressive means, one in five a mean
    tension of up to 3 scale with a small deviator (the apex region)."""
    out = []
    for i in range(n):
        if i % 5 == 4:
            s = rng.normal(0, 0.1 * scale, 6)
            s[:3] += rng.uniform(0.0, 3.0 * scale)
        else:
            s = rng.normal(0, scale, 6)
            s[:3] += rng.normal(-scale, scale)
        out.append(s)
    return out


def test_eigensolver_matches_lapack():
    rng = np.random.default_rng(5)
    for _ in range(300):
        s6 = rng.normal(0, 1e4, 6)
        lam, V = oracle.eig_sym3(s6)
        S = np.array([[s6[0], s6[3], s6[5]], [s6[3], s6[1], s6[4]], [s6[5], s6[4], s6[2]]])
        assert np.allclose(np.sort(lam), np.linalg.eigvalsh(S), rtol=0, atol=1e-10 * np.abs(S).max())
        assert np.allclose(S @ V, V * lam[None, :], atol=1e-9 * np.abs(S).max())
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-13)


def test_elastic_trial_is_unchanged():
    phi, c = math.radians(30), 5e3
    rng = np.random.default_rng(6)
    for s in random_trials(rng, 300, 2e4):
        if mc_planes(principal(s), phi, c).max() <= 0:
            out, br, d = oracle.mc_return(E, NU, phi, 0.0, c, s)
            assert br == 0 and np.array_equal(out, s) and d == 0.0


@pytest.mark.parametrize("c", [0.0, 10e3])
def test_associated_return_is_closest_point(c):
    phi = math.radians(30)
    rng = np.random.default_rng(7 + int(c))
    seen = set()
    for s in random_trials(rng, 400, 3e4):
        sp = principal(s)
        if mc_planes(sp, phi, c).max() <= 0:
            continue
        out, br, _ = oracle.mc_return(E, NU, phi, phi, c, s)
        seen.add(br)
        got = principal(out)
        # closest admissible point in the complementary-energy norm
        A = []
        for i in range(3):
            for j in range(3):
                if i != j:
                    row = np.zeros(3)
                    row[i] = 1 + math.sin(phi)
                    row[j] = -(1 - math.sin(phi))
                    A.append(row)
        A = np.array(A)
        b = 2 * c * math.cos(phi)
        scale = np.abs(sp).max() + c
        fun = lambda y: 0.5 * (sp - y * scale) @ CMAT @ (sp - y * scale) * E / scale ** 2
        jac = lambda y: -(CMAT @ (sp - y * scale)) * E / scale
        cons = {"type": "ineq", "fun": lambda y: b / scale - A @ y, "jac": lambda y: -A}
        res = minimize(fun, got / scale, jac=jac, constraints=[cons], method="SLSQP",
                       options=dict(ftol=1e-16, maxiter=500))
        best = np.sort(res.x * scale)[::-1]
        assert np.allclose(got, best, atol=2e-6 * scale), (br, got, best)
        assert mc_planes(got, phi, c).max() <= 1e-9 * scale
    assert {1, 2, 3, 4} <= seen, seen


def test_nonassociated_flow_direction():
    phi, psi, c = math.radians(30), 0.0, 2e3
    sp_ = math.sin(psi)
    Na = np.array([1 + sp_, 0, -(1 - sp_)])
    Nb = np.array([0, 1 + sp_, -(1 - sp_)])
    Nc = np.array([1 + sp_, -(1 - sp_), 0])
    rng = np.random.default_rng(8)
    seen = set()
    for s in random_trials(rng, 400, 3e4):
        sp = principal(s)
        if mc_planes(sp, phi, c).max() <= 0:
            continue
        out, br, d = oracle.mc_return(E, NU, phi, psi, c, s)
        seen.add(br)
        got = principal(out)
        assert mc_planes(got, phi, c).max() <= 1e-9 * (np.abs(sp).max() + c)
        if br == 4:
            assert np.allclose(got, c / math.tan(phi), rtol=1e-12)
            continue
        dep = CMAT @ (sp - got)      # plastic strain in principal axes
        basis = {1: [Na], 2: [Na, Nb], 3: [Na, Nc]}[br]
        B = np.stack(basis, axis=1)
        coef, resid = nnls(B, dep)
        assert resid <= 1e-9 * np.abs(dep).max()
        assert np.all(coef >= 0)
        assert d == pytest.approx(math.sqrt(2 / 3 * dep @ dep), rel=1e-9)
    assert {1, 2, 3, 4} <= seen, seen


@pytest.mark.parametrize("c", [0.0, 7e3])
def test_hydrostatic_tension_goes_to_apex(c):
    phi = math.radians(30)
    p = 5e4
    out, br, _ = oracle.mc_return(E, NU, phi, 0.0, c, [p, p, p, 0, 0, 0])
    assert br == 4
    assert np.allclose(out, [c / math.tan(phi)] * 3 + [0, 0, 0], rtol=1e-12, atol=1e-9)


def test_triaxial_compression_reaches_rankine_ratio():
    """Strain-driven drained triaxial compression at constant lateral stress."""
    phi = math.radians(30)
    mat = oracle.Material(model=oracle.MOHR_COULOMB, E=E, nu=NU, rho=1800.0, phi=phi, c=0.0, psi=0.0)
    p0 = 1e5
    sig = np.array([-p0, -p0, -p0, 0, 0, 0], dtype=float)
    dez = -1e-5
    first_slope = None
    for it in range(10000):
        # find the lateral strain keeping sig_xx = sig_yy = -p0 (secant iterations)
        def resid(e):
            s, _ = oracle.stress_update(mat, 0.0, sig, [e, e, dez, 0, 0, 0])
            return s[0] + p0
        e0, e1 = 0.0, -NU * dez
        r0, r1 = resid(e0), resid(e1)
        for _ in range(40):
            if r1 == r0:
                break
            e2 = e1 - r1 * (e1 - e0) / (r1 - r0)
            e0, r0, e1, r1 = e1, r1, e2, resid(e2)
            if abs(r1) < 1e-9 * p0:
                break
        new, _ = oracle.stress_update(mat, 0.0, sig, [e1, e1, dez, 0, 0, 0])
        if first_slope is None:
            first_slope = (new[2] - sig[2]) / dez
        sig = new
        if it * abs(dez) > 0.05:
            break
    assert first_slope == pytest.approx(E, rel=1e-9)
    kp = (1 + math.sin(phi)) / (1 - math.sin(phi))
    assert sig[2] / sig[0] == pytest.approx(kp, rel=1e-9)
    assert kp == pytest.approx(3.0, rel=1e-12)
