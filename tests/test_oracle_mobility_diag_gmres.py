"""Pins of the oracle's mobility, beta, Jacobi diagonal and GMRES."""
import math
import os

import numpy as np
import pytest

from oracle import blocks, diag, gmres, mobility
from oracle.fields import Problem, State
from tests.helpers import desc_small, state_of
from workloads import node_coords

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _steady(x):
    return State(x.copy(), x.copy(), np.zeros_like(x))


def test_appendix_a_l2_projection_values():
    """Appendix A: lumped L2-projection of the derivative 2x of x^2 (evaluated at the
    quadrature points, as in the worked example) on [0,2] and [-1,3] (golden file,
    values printed to 3 decimals), reproduced in 3D with a field of x only."""
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "appendix_a_l2_projection.txt"))
            if l.strip() and not l.startswith("#")]
    for lo, hi in sorted({(r[0], r[1]) for r in rows}):
        n = int(round(hi - lo))
        d = desc_small(n=(n, 1, 1), L=(hi - lo, 1.0, 1.0), dirichlet=False, n_solid=0)
        pb = Problem(d)
        X = node_coords(d)
        x = X[0] + lo
        xq = pb.mesh.val(x)  # exact: x is linear
        g = mobility.l2_project(pb, 2.0 * xq)
        for r in rows:
            if (r[0], r[1]) != (lo, hi):
                continue
            sel = np.isclose(x, r[2])
            assert np.allclose(np.round(g[sel], 3), r[3], atol=1e-12)


def test_mobility_closed_form_linear_fields():
    """Linear phi (inside the band) and linear v = A x: q = a^T A a / |a|^2 exactly
    at every quadrature point and node, so gamma = |q| / eta."""
    d = desc_small(n=(3, 4, 3), dirichlet=False, n_solid=0)
    pb = Problem(d)
    X = node_coords(d)
    a = np.array([0.2, -0.1, 0.15])
    A = np.array([[0.3, 1.0, -0.2], [0.1, -0.5, 0.4], [0.7, 0.2, 0.9]])
    x = np.zeros((d.ncomp, d.nn))
    x[0:3] = A @ X
    x[4] = -0.3 + a @ X
    q = a @ A @ a / (a @ a)
    g = mobility.mobility(pb, _steady(x), 0)
    assert g == pytest.approx(abs(q) / d.eta, rel=1e-13)


def test_mobility_band_and_projection_by_brute_force():
    """Nodal values by explicit element loops (sum over elements of quadrature sums
    of N_p q and N_p), the band |phi_p| <= 0.9, RMS over band nodes, 1/eta."""
    d = desc_small(n=(2, 3, 2), dirichlet=False, n_solid=0)
    pb = Problem(d)
    st = state_of(d, 31, phi_range=1.0)
    wave = 1.4 * np.sin(np.arange(d.nn) * 0.7)
    st.x[4], st.xn[4] = wave, 0.9 * wave
    m = pb.mesh
    xa = pb.at_alpha(st)
    num = np.zeros(m.nn)
    den = np.zeros(m.nn)
    for e in range(m.ne):
        nodes = m.conn[e]
        for qp in range(8):
            gphi = sum(xa[4][nodes[a]] * m.dN[qp, a] for a in range(8))
            L = np.array([[sum(xa[j][nodes[a]] * m.dN[qp, a, k] for a in range(8)) for k in range(3)]
                          for j in range(3)])
            n2 = gphi @ gphi
            q = 0.0 if n2 < 1e-30 else gphi @ L @ gphi / n2
            for a in range(8):
                num[nodes[a]] += m.wq * m.N[qp, a] * q
                den[nodes[a]] += m.wq * m.N[qp, a]
    band = np.abs(xa[4]) <= 0.9
    assert 0 < band.sum() < m.nn
    expect = math.sqrt((np.abs(num / den)[band] ** 2).mean()) / d.eta
    assert mobility.mobility(pb, st, 0) == pytest.approx(expect, rel=1e-12)


def test_mobility_zero_cases():
    d = desc_small(n=(2, 2, 2), dirichlet=False, n_solid=0)
    pb = Problem(d)
    x = np.zeros((d.ncomp, d.nn))
    x[4] = 0.95  # no node in the band
    x[0:3] = np.random.default_rng(0).normal(size=(3, d.nn))
    assert mobility.mobility(pb, _steady(x), 0) == 0.0
    x[4] = np.linspace(-0.5, 0.5, d.nn)
    x[0:3] = 0.0  # v = 0
    assert mobility.mobility(pb, _steady(x), 0) == 0.0


@pytest.mark.parametrize("c", [0.4, -0.7, 1.3])
def test_beta_constant_phi(c):
    """Uniform phi = c: beta = (c^3 - c) / (|c^2 - 1|/2) = 2 c sign(c^2 - 1)."""
    d = desc_small(n=(2, 2, 3), dirichlet=False, n_solid=0)
    pb = Problem(d)
    x = np.zeros((d.ncomp, d.nn))
    x[4] = c
    assert mobility.beta(pb, _steady(x), 0) == pytest.approx(2 * c * np.sign(c * c - 1), rel=1e-13)


def test_beta_linear_phi_closed_form():
    """phi = a + b x on [0, 1] with |phi| < 1: Gauss quadrature is exact for the
    polynomial integrands, beta = int (phi^3 - phi) / int (1 - phi^2)/2."""
    d = desc_small(n=(4, 1, 1), dirichlet=False, n_solid=0)
    pb = Problem(d)
    X = node_coords(d)
    a, b = -0.3, 0.5
    x = np.zeros((d.ncomp, d.nn))
    x[4] = a + b * X[0]
    # int_0^1 phi^k dx = ((a+b)^{k+1} - a^{k+1}) / ((k+1) b)
    I = lambda k: ((a + b) ** (k + 1) - a ** (k + 1)) / ((k + 1) * b)
    expect = (I(3) - I(1)) / (0.5 * (I(0) - I(2)))
    assert mobility.beta(pb, _steady(x), 0) == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("block", ["ns", ("ac", 1), ("b", 0)])
def test_diagonal_by_probing_equals_unit_vector_products(block):
    """Probing by 27 colours equals e_i^T J e_i computed one unit vector at a time."""
    d = desc_small(n=(2, 2, 3), n_fluid=1, n_solid=1)
    pb = Problem(d)
    st = state_of(d, 17)
    coeffs = {"gamma": {1: 0.4}, "beta": {1: 0.1}}
    dg = diag.block_diagonal(pb, st, block, coeffs)
    n = dg.size
    for i in range(0, n, 3):
        e = np.zeros(n)
        e[i] = 1.0
        assert dg[i] == blocks.jvp(pb, st, block, e, coeffs)[i]


def test_gmres_matches_dense_solve():
    """GMRES on the assembled NS Jacobian of a tiny mesh equals a dense LU solve."""
    d = desc_small(n=(2, 2, 2), n_fluid=1, n_solid=1)
    pb = Problem(d)
    st = state_of(d, 19)
    n = 4 * d.nn
    A = np.stack([blocks.jvp(pb, st, "ns", np.eye(n)[i]) for i in range(n)], axis=1)
    b = np.random.default_rng(3).normal(size=n)
    dg = np.diag(A)
    x, it, rel = gmres.gmres(lambda u: A @ u, b, 1.0 / dg, m=10, rtol=1e-12, max_iter=500)
    xd = np.linalg.solve(A, b)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9
    assert it > 10  # restarted at least once


def test_gmres_laplacian_against_scipy():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    n = 200
    A = sp.diags([-np.ones(n - 1), 2.5 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    b = np.random.default_rng(0).normal(size=n)
    x, it, rel = gmres.gmres(lambda u: A @ u, b, None, m=30, rtol=1e-10, max_iter=2000)
    assert rel <= 1e-10
    xs = spl.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xs) <= 10 * 1e-10 * np.linalg.norm(xs)  # cond(A) <= 9
