"""Pins of the oracle's shape functions and particle-to-grid transfer.

The linear quad/hex shape functions (CODE OVERVIEW: linear mapping functions
of the 4-node quadrilateral and 8-node hexahedron) are pinned by the
properties that define a linear Lagrange element -- partition of unity,
linear completeness, Kronecker delta at the nodes -- and the whole P2G
transfer (INTRODUCTION: particle -> node mapping) by a brute-force double
loop over all particle-node pairs that evaluates the global tent functions
N_i(x) = prod_k max(0, 1 - |x_k - X_ik| / h) directly from coordinates, a
formulation independent of the oracle's cell/natural-coordinate one.
"""
import numpy as np
import pytest

import oracle
from paper_1909_13380_gb300 import workloads as W


@pytest.mark.parametrize("dim", [2, 3])
def test_partition_of_unity_and_gradient_sum(dim):
    rng = np.random.default_rng(1)
    for _ in range(200):
        xi = rng.uniform(-1, 1, dim)
        N, dN = oracle.shape(dim, xi)
        nn = 1 << dim
        assert abs(N[:nn].sum() - 1.0) < 1e-15
        assert np.all(np.abs(dN[:nn].sum(axis=0)) < 1e-15)
        assert np.all(N[nn:] == 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_completeness(dim):
    rng = np.random.default_rng(2)
    nn = 1 << dim
    nodes = np.array([[1.0 if (a >> k) & 1 else -1.0 for k in range(dim)] for a in range(nn)])
    for _ in range(100):
        xi = rng.uniform(-1, 1, dim)
        N, dN = oracle.shape(dim, xi)
        # sum_a N_a xi^a = xi ; sum_a dN_a/dxi_k xi^a_j = delta_jk
        assert np.allclose(N[:nn] @ nodes, xi, atol=1e-15)
        assert np.allclose(nodes.T @ dN[:nn, :dim], np.eye(dim), atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_kronecker_delta_at_nodes(dim):
    nn = 1 << dim
    for b in range(nn):
        xi = [1.0 if (b >> k) & 1 else -1.0 for k in range(dim)]
        N, _ = oracle.shape(dim, xi)
        expect = np.zeros(nn)
        expect[b] = 1.0
        assert np.array_equal(N[:nn], expect)


def test_locate_rule():
    mesh = oracle.Mesh(dim=3, n=(4, 3, 2), h=0.5, origin=(1.0, -1.0, 0.0))
    # exactly on an interior face: the higher cell (floor)
    st, c, xi = oracle.locate_one(mesh, [1.5, -1.0, 0.25])
    assert st == oracle.OK and list(c) == [1, 0, 0] and xi[0] == -1.0 and xi[1] == -1.0
    # the upper mesh bound has left the mesh; so has anything below the origin
    assert oracle.locate_one(mesh, [3.0, 0.0, 0.5])[0] == oracle.LEFT_MESH
    assert oracle.locate_one(mesh, [2.999999, 0.0, 0.5])[0] == oracle.OK
    assert oracle.locate_one(mesh, [0.9999999, 0.0, 0.5])[0] == oracle.LEFT_MESH
    assert oracle.locate_one(mesh, [float("nan"), 0.0, 0.5])[0] == oracle.LEFT_MESH


def brute_force_p2g(dim, ncells, h, g, pos, vel, sig, m, vol):
    """Double loop over (node, particle) with global tent functions."""
    shape_n = [ncells[k] + 1 for k in range(dim)]
    grids = np.meshgrid(*[np.arange(s) for s in shape_n[::-1]], indexing="ij")
    X = np.stack([gk.ravel() for gk in grids[::-1]], axis=1) * h          # node coords, x fastest
    nn = X.shape[0]
    nm, nP, nf = np.zeros(nn), np.zeros((nn, 3)), np.zeros((nn, 3))
    S = np.zeros((pos.shape[0], 3, 3))
    vo = [(0, 0, 0), (1, 1, 1), (2, 2, 2), (0, 1, 3), (1, 2, 4), (0, 2, 5)]
    for j, k, c in vo:
        S[:, j, k] = S[:, k, j] = sig[:, c]
    for i in range(nn):
        r = (pos - X[i]) / h                                   # (np, dim)
        w = np.maximum(0.0, 1.0 - np.abs(r))
        N = np.prod(w, axis=1)
        grad = np.zeros((pos.shape[0], 3))
        for k in range(dim):
            dk = np.where(np.abs(r[:, k]) < 1.0, -np.sign(r[:, k]) / h, 0.0)
            others = np.prod(np.delete(w, k, axis=1), axis=1) if dim > 1 else 1.0
            grad[:, k] = dk * others
        nm[i] = np.sum(N * m)
        nP[i, :dim] = (N * m) @ vel[:, :dim]
        fint = -np.einsum("p,pjk,pk->j", vol, S, grad)
        nf[i] = fint + np.sum(N * m) * np.asarray(g)
        nf[i, dim:] = 0.0
    return nm, nP, nf


@pytest.mark.parametrize("dim", [2, 3])
def test_p2g_matches_brute_force(dim):
    ncells = (5, 4, 3)[:dim] + (1,) * (3 - dim)
    h = 0.25
    pos, vel, sig, vol = W.random_particles(ncells, h, 60, seed=11 + dim, dim=dim, margin=0)
    g = (0.3, -9.81, 1.7) if dim == 3 else (0.3, -9.81, 0.0)
    mesh = oracle.Mesh(dim=dim, n=ncells, h=h, g=g)
    st = oracle.State.create(pos, vel, vol, rho=1500.0, sig0=sig)
    o = oracle.Oracle(mesh, oracle.Material(), st)
    nm, nP, nf = o.p2g()
    bm, bP, bf = brute_force_p2g(dim, ncells, h, g, st.x[:, :dim], st.v, st.sig, st.m, st.vol)
    assert np.allclose(nm, bm, rtol=1e-13, atol=1e-13 * np.abs(bm).max())
    assert np.allclose(nP, bP, rtol=1e-12, atol=1e-12 * np.abs(bP).max())
    assert np.allclose(nf, bf, rtol=1e-12, atol=1e-12 * np.abs(bf).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_p2g_conserves_mass_momentum_and_internal_force(dim):
    ncells = (6, 5, 4)[:dim] + (1,) * (3 - dim)
    h = 0.1
    pos, vel, sig, vol = W.random_particles(ncells, h, 500, seed=21 + dim, dim=dim, margin=0)
    mesh = oracle.Mesh(dim=dim, n=ncells, h=h, g=(0.0, 0.0, 0.0))
    st = oracle.State.create(pos, vel, vol, rho=2000.0, sig0=sig)
    o = oracle.Oracle(mesh, oracle.Material(), st)
    nm, nP, nf = o.p2g()
    M = st.m.sum()
    assert abs(nm.sum() - M) <= 1e-14 * M
    assert np.allclose(nP.sum(axis=0), (st.m[:, None] * st.v).sum(axis=0), rtol=1e-13, atol=1e-13 * M)
    # internal forces are self-equilibrated: sum_a grad N_a = 0
    assert np.all(np.abs(nf.sum(axis=0)) <= 1e-10 * np.abs(nf).sum())
    # gravity only adds m_i g at every node
    g = np.array([0.5, -9.81, 2.0 if dim == 3 else 0.0])
    o.mesh.g = tuple(g)
    nm2, _, nf2 = o.p2g()
    assert np.allclose(nf2 - nf, nm2[:, None] * g[None, :], rtol=1e-12, atol=1e-12 * np.abs(nf2).max())
