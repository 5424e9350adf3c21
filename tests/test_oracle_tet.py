"""Pins of the oracle's linear-tetrahedron variant (oracle/tet.py): mesh conformity and
volume, quadrature exactness, reproduction of linear fields, the reference metric, the
Couette patch and rigid-motion tests of the weak forms, and the Jacobian-vector product
against finite differences of the residual."""
import itertools

import numpy as np
import pytest

from oracle import ac, cgt, ns
from oracle.fields import State
from oracle.tet import QBARY, TetMesh, TetProblem
from tests.helpers import desc_small, state_of


def _desc(n=(3, 4, 2), L=(1.0, 1.3, 0.7), **kw):
    return desc_small(n=n, L=L, **kw)


@pytest.mark.parametrize("jitter", [0.0, 0.25])
def test_mesh_is_conforming_with_the_box_volume(jitter):
    d = _desc()
    m = TetMesh(d, jitter=jitter, seed=1)
    assert (m.vol > 0).all()
    assert m.vol.sum() == pytest.approx(d.lx * d.ly * d.lz, rel=1e-13)
    faces = {}
    for e in range(m.ne):
        for f in itertools.combinations(sorted(m.conn[e]), 3):
            faces[f] = faces.get(f, 0) + 1
    assert max(faces.values()) == 2
    boundary = [f for f, c in faces.items() if c == 1]
    i, j, k = m.ijk()
    on = lambda nodes, axis, val: all((i, j, k)[axis][n] == val for n in nodes)
    for f in boundary:  # every unshared face lies on a box face
        assert any(on(f, a, 0) or on(f, a, (d.nx, d.ny, d.nz)[a]) for a in range(3))
    # two triangles per boundary cell face
    nb = 2 * 2 * (d.nx * d.ny + d.ny * d.nz + d.nx * d.nz)
    assert len(boundary) == nb


def test_quadrature_is_exact_for_quadratics_and_reproduces_linear_fields():
    d = _desc()
    m = TetMesh(d, jitter=0.3, seed=2)
    X = m.X
    # int x_i x_j over the box
    for a, b in [(0, 0), (0, 1), (1, 2), (2, 2)]:
        got = m.integrate_scalar(m.val(X[a]) * m.val(X[b]))
        L = (d.lx, d.ly, d.lz)
        V = L[0] * L[1] * L[2]
        exact = V * (L[a] ** 2 / 3.0 if a == b else L[a] * L[b] / 4.0)
        assert got == pytest.approx(exact, rel=1e-13)
    u = 0.3 + 1.2 * X[0] - 0.7 * X[1] + 2.5 * X[2]
    g = m.grad(u)
    assert np.abs(g - np.array([1.2, -0.7, 2.5])).max() < 1e-12
    # the quadrature points' values are the field at the points
    xq = np.einsum("qa,dea->deq", QBARY, X[:, m.conn])
    assert np.abs(m.val(u) - (0.3 + 1.2 * xq[0] - 0.7 * xq[1] + 2.5 * xq[2])).max() < 1e-13


def test_reference_metric_is_the_identity_on_the_unit_right_tetrahedron():
    """G = sum_k grad xi_k grad xi_k^T: the identity on the reference element, 1/s^2 on
    it scaled by s."""
    d = desc_small(n=(1, 1, 1), L=(1.0, 1.0, 1.0))
    m = TetMesh(d)
    # the tetrahedron 0 -> e_x -> e_x + e_y -> 7 maps (xi_1, xi_2, xi_3) linearly; check the
    # definition on every element against grad(lambda_k) from a direct solve
    for e in range(m.ne):
        P = m.X[:, m.conn[e]].T  # (4, 3)
        A = np.hstack([np.ones((4, 1)), P])  # lambda = A^{-T} [1, x]
        grads = np.linalg.inv(A)[1:, :].T  # (4a, 3)
        assert np.abs(grads - m.dNe[e]).max() < 1e-13
        G = sum(np.outer(grads[k], grads[k]) for k in (1, 2, 3))
        assert np.abs(G - m.G[e]).max() < 1e-12
    d2 = desc_small(n=(1, 1, 1), L=(2.0, 2.0, 2.0))
    assert np.allclose(TetMesh(d2).G, m.G / 4.0, rtol=1e-13)


def _couette(d, pb):
    nn = d.nn
    X = pb.mesh.X
    x = np.zeros((d.ncomp, nn))
    x[0] = X[2]
    x[3] = 0.4
    x[4:4 + d.n_phase] = -1.0
    x[4] = 1.0  # one fluid
    base = 4 + d.n_phase
    for s in range(d.n_solid):
        x[base + 6 * s: base + 6 * s + 3] = 1.0
    return State(x.copy(), x.copy(), np.zeros_like(x))


def test_couette_patch_interior_rows_vanish():
    d = _desc(n=(4, 3, 4), dirichlet=False, n_fluid=1, n_solid=1)
    pb = TetProblem(d, jitter=0.2, seed=3)
    st = _couette(d, pb)
    r = ns.ns_residual(pb, st)
    i, j, k = pb.mesh.ijk()
    inner = (i > 0) & (i < d.nx) & (j > 0) & (j < d.ny) & (k > 0) & (k < d.nz)
    scale = np.abs(ns.ns_residual(pb, State(st.x * 1.7 + 0.1, st.xn, st.xdn))).max()
    assert np.abs(r[:, inner]).max() <= 1e-12 * scale


def test_rigid_motion_keeps_b_identity():
    d = _desc(n=(3, 3, 3), dirichlet=False, n_fluid=1, n_solid=1)
    pb = TetProblem(d, jitter=0.2, seed=4)
    X = pb.mesh.X
    x = np.zeros((d.ncomp, d.nn))
    w = np.array([0.3, -0.5, 0.2])
    c = np.array([0.5, 0.6, 0.3])
    r = X - c[:, None]
    v = np.cross(w, r.T).T + np.array([0.1, 0.2, -0.3])[:, None]
    x[0:3] = v
    x[4] = 0.0
    x[5] = 0.3
    x[6:9] = 1.0
    st = State(x.copy(), x.copy(), np.zeros_like(x))
    res = cgt.cgt_residual(pb, st, 0)
    assert np.abs(res).max() < 1e-13


@pytest.mark.parametrize("block", ["ns", "ac"])
def test_jvp_matches_finite_differences(block):
    d = _desc(n=(3, 2, 3), n_fluid=1, n_solid=1)
    pb = TetProblem(d, jitter=0.25, seed=5)
    st = state_of(d, 6)
    rng = np.random.default_rng(7)
    if block == "ns":
        dx = rng.normal(size=(4, d.nn))
        J = ns.ns_jvp(pb, st, dx, elastic_aug=False)

        def R(x):
            return ns.ns_residual(pb, State(x, st.xn, st.xdn), coef=st)

        comps = slice(0, 4)
    else:
        dx = rng.normal(size=(1, d.nn))
        J = ac.ac_jvp(pb, st, 1, 0.4, 0.1, dx[0])[None]

        def R(x):
            return ac.ac_residual(pb, State(x, st.xn, st.xdn), 1, 0.4, 0.1, coef=st)[None]

        comps = slice(5, 6)
    h = 1e-6 * np.linalg.norm(st.x[comps]) / np.linalg.norm(dx)
    xp, xm = st.x.copy(), st.x.copy()
    xp[comps] += h * dx
    xm[comps] -= h * dx
    fd = (R(xp) - R(xm)) / (2 * h)
    assert np.linalg.norm(J - fd) <= 1e-7 * np.linalg.norm(J)


def test_box_mesh_generator_orientation_and_reproducibility():
    """workloads.tet_box_mesh (the seeded input shared by the oracle and the GPU side): every
    element positively oriented, six per cell, the same mesh for the same seed, a different
    jitter for another seed, boundary nodes never moved."""
    from workloads import tet_box_mesh
    d = _desc(n=(3, 2, 4))
    X1, c1 = tet_box_mesh(d, 0.3, seed=5)
    X2, c2 = tet_box_mesh(d, 0.3, seed=5)
    X3, _ = tet_box_mesh(d, 0.3, seed=6)
    assert c1.shape == (6 * d.nx * d.ny * d.nz, 4)
    assert np.array_equal(X1, X2) and np.array_equal(c1, c2)
    assert not np.array_equal(X1, X3)
    e1, e2, e3 = (X1[:, c1[:, a]] - X1[:, c1[:, 0]] for a in (1, 2, 3))
    det = np.einsum("ie,ie->e", e1, np.cross(e2.T, e3.T).T)
    assert (det > 0).all()
    X0, _ = tet_box_mesh(d, 0.0)
    n = np.arange(d.nn)
    i, j, k = n % (d.nx + 1), (n // (d.nx + 1)) % (d.ny + 1), n // ((d.nx + 1) * (d.ny + 1))
    bnd = (i == 0) | (i == d.nx) | (j == 0) | (j == d.ny) | (k == 0) | (k == d.nz)
    assert np.array_equal(X1[:, bnd], X0[:, bnd])
