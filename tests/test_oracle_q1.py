"""Pins of the oracle's Q1 element: shape functions, quadrature, assembly."""
import numpy as np
import pytest

from oracle.q1 import Q1Mesh, corner_signs, gauss_points, shape_gradients, shape_values


def test_shape_kronecker_at_corners():
    N = shape_values(corner_signs())
    assert np.array_equal(N, np.eye(8))


def test_partition_of_unity():
    xi = np.random.default_rng(0).uniform(-1, 1, size=(20, 3))
    assert np.allclose(shape_values(xi).sum(1), 1.0, atol=1e-15)
    assert np.allclose(shape_gradients(xi, (0.3, 0.5, 0.7)).sum(1), 0.0, atol=1e-14)


@pytest.mark.parametrize("n", [(2, 3, 4), (5, 2, 3)])
def test_linear_fields_reproduced(n):
    """Q1 reproduces linear fields: values at quadrature points equal the field at
    their physical coordinates and gradients equal the exact gradient."""
    m = Q1Mesh(*n, 1.3, 0.7, 2.1)
    i, j, k = m.ijk()
    X = np.stack([i * m.h[0], j * m.h[1], k * m.h[2]])
    a, b = 0.37, np.array([1.1, -2.3, 0.7])
    u = a + b @ X
    g = m.grad(u)
    assert np.allclose(g, b[None, None, :], atol=1e-12)
    # physical coordinates of quadrature points
    xi = gauss_points()
    xq = np.stack([m.val(X[d]) for d in range(3)])
    e0 = m.conn[:, 0]
    for d in range(3):
        expect = X[d][e0][:, None] + (1.0 + xi[None, :, d]) * m.h[d] / 2.0
        assert np.allclose(xq[d], expect, atol=1e-13)
    assert np.allclose(m.val(u), a + np.einsum("d,deq->eq", b, xq), atol=1e-12)


def test_quadrature_exact_for_trilinear_times_trilinear():
    """int x^2 y z^3 over [0,1]x[0,2]x[0,1] is integrated exactly (degree <= 3 per axis)."""
    m = Q1Mesh(3, 4, 2, 1.0, 2.0, 1.0)
    xq = np.stack([m.val(c) for c in _coords(m)])
    f = xq[0] ** 2 * xq[1] * xq[2] ** 3
    exact = (1.0 / 3.0) * (4.0 / 2.0) * (1.0 / 4.0)
    assert m.integrate_scalar(f) == pytest.approx(exact, rel=1e-14)


def test_assembly_sums_to_volume_and_lumped_mass_closed_form():
    m = Q1Mesh(3, 3, 3, 1.5, 1.5, 1.5)
    r = m.integrate(np.ones((m.ne, 8)))
    assert r.sum() == pytest.approx(1.5 ** 3, rel=1e-14)
    h3 = m.h[0] * m.h[1] * m.h[2]
    i, j, k = m.ijk()
    nb = (i == 0) | (i == 3)
    nb = nb.astype(int) + ((j == 0) | (j == 3)) + ((k == 0) | (k == 3))
    # int N_a = h^3 / 2^(number of boundary directions)
    assert np.allclose(r, h3 / 2.0 ** nb, rtol=1e-14)


def test_gradient_integration_by_parts():
    """sum_a u_a int grad N_a . g = int grad u . g for constant g (test/trial symmetry)."""
    m = Q1Mesh(3, 2, 2, 1.0, 1.0, 1.0)
    u = np.random.default_rng(1).normal(size=m.nn)
    g = np.zeros((m.ne, 8, 3))
    g[..., 1] = 0.7
    lhs = u @ m.integrate(None, g)
    rhs = m.integrate_scalar((m.grad(u) * g).sum(-1))
    assert lhs == pytest.approx(rhs, rel=1e-13)


def _coords(m):
    i, j, k = m.ijk()
    return [i * m.h[0], j * m.h[1], k * m.h[2]]
