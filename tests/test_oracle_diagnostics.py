"""Pins of the oracle's diagnostics (Section 5.2 centre of mass, Appendix C point
tracking): closed forms for linear fields, an element-by-element analytic integral,
symmetry, and the exactness of trilinear interpolation for linear velocity fields."""
import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle.fields import Problem
from tests.helpers import desc_small


def _problem(n=(5, 4, 6), L=(1.0, 0.8, 1.2), dt=0.01):
    return Problem(desc_small(n=n, L=L, n_fluid=1, n_solid=1, dt=dt))


def _state_with_alpha(pb, alpha):
    x = np.zeros((pb.desc.ncomp, pb.mesh.nn))
    x[pb.phi_comp(pb.solids[0])] = 2.0 * alpha - 1.0
    return x


def test_center_of_mass_of_a_linear_indicator_closed_form():
    """alpha = a + b x + c y: the centre of mass has a closed form over the box, and
    the 2x2x2 Gauss rule integrates x alpha exactly."""
    pb = _problem()
    d = pb.desc
    X = dg.node_xyz(pb)
    a, b, c = 0.3, 0.25, -0.2
    x = _state_with_alpha(pb, a + b * X[0] + c * X[1])
    Lx, Ly, Lz = d.lx, d.ly, d.lz
    mass = Lx * Ly * Lz * (a + b * Lx / 2 + c * Ly / 2)
    mx = Lz * (a * Lx ** 2 / 2 * Ly + b * Lx ** 3 / 3 * Ly + c * Lx ** 2 / 2 * Ly ** 2 / 2)
    my = Lz * (a * Ly ** 2 / 2 * Lx + b * Lx ** 2 / 2 * Ly ** 2 / 2 + c * Ly ** 3 / 3 * Lx)
    mz = Lz ** 2 / 2 * (a * Lx * Ly + b * Lx ** 2 / 2 * Ly + c * Lx * Ly ** 2 / 2)
    np.testing.assert_allclose(dg.center_of_mass(pb, x, 0), [mx / mass, my / mass, mz / mass], rtol=1e-13)


def test_center_of_mass_matches_elementwise_analytic_integrals():
    """Random nodal indicator: per element, int x N_a = h^3 (x0/8 + h I(a)/4) with
    I = 1/6 for the lower and 1/3 for the upper corner along the axis (1D integrals
    of (1 - t) and t against t); the sums give the same centre to rounding."""
    pb = _problem(n=(3, 4, 2), L=(0.9, 1.1, 0.7))
    m = pb.mesh
    rng = np.random.default_rng(3)
    alpha = rng.uniform(0.0, 1.0, size=m.nn)
    x = _state_with_alpha(pb, alpha)
    X = dg.node_xyz(pb)
    vol = m.h[0] * m.h[1] * m.h[2]
    mass, mom = 0.0, np.zeros(3)
    for e in range(m.ne):
        for aa in range(8):
            al = alpha[m.conn[e, aa]]
            mass += vol * al / 8.0
            s = [aa & 1, (aa >> 1) & 1, (aa >> 2) & 1]
            for dd in range(3):
                x0 = X[dd, m.conn[e, 0]]
                Ia = 1.0 / 3.0 if s[dd] else 1.0 / 6.0
                mom[dd] += vol * al * (x0 / 8.0 + m.h[dd] * Ia / 4.0)
    np.testing.assert_allclose(dg.center_of_mass(pb, x, 0), mom / mass, rtol=1e-13)


def test_center_of_mass_of_a_centred_sphere_is_the_box_centre():
    pb = _problem(n=(6, 6, 6), L=(1.0, 1.0, 1.0))
    X = dg.node_xyz(pb)
    r = np.sqrt(((X - 0.5) ** 2).sum(0))
    x = np.zeros((pb.desc.ncomp, pb.mesh.nn))
    x[pb.phi_comp(pb.solids[0])] = np.tanh((0.3 - r) / 0.1)
    np.testing.assert_allclose(dg.center_of_mass(pb, x, 0), [0.5, 0.5, 0.5], atol=1e-14)


def _linear_velocity(pb, A, b):
    X = dg.node_xyz(pb)
    x = np.zeros((pb.desc.ncomp, pb.mesh.nn))
    for k in range(3):
        x[k] = A[k] @ X + b[k]
    return x


def test_interpolation_reproduces_linear_velocity_fields():
    """Trilinear interpolation is exact for v = A p + b with a full A (a swapped corner
    order or a mis-scaled local coordinate would not be)."""
    pb = _problem()
    rng = np.random.default_rng(1)
    A = rng.normal(size=(3, 3))
    b = rng.normal(size=3)
    x = _linear_velocity(pb, A, b)
    d = pb.desc
    pts = rng.uniform(0.0, 1.0, size=(200, 3)) * [d.lx, d.ly, d.lz]
    np.testing.assert_allclose(dg.interpolate_velocity(pb, x, pts), pts @ A.T + b, rtol=1e-12, atol=1e-12)


def test_interpolation_at_nodes_faces_and_outside():
    pb = _problem()
    m = pb.mesh
    rng = np.random.default_rng(2)
    x = np.zeros((pb.desc.ncomp, m.nn))
    x[0:3] = rng.normal(size=(3, m.nn))
    X = dg.node_xyz(pb)
    # at the nodes (including the upper box faces): the nodal values
    nodes = np.arange(m.nn)
    np.testing.assert_allclose(dg.interpolate_velocity(pb, x, X[:, nodes].T), x[0:3, nodes].T, atol=1e-13)
    # on an interior face: the limit from both sides
    p = np.array([[2 * m.h[0], 0.37, 0.51]])
    for eps in (1e-11, -1e-11):
        q = p + [eps, 0.0, 0.0]
        np.testing.assert_allclose(dg.interpolate_velocity(pb, x, q), dg.interpolate_velocity(pb, x, p), atol=1e-9)
    # outside the box: the value at the clamped point
    d = pb.desc
    out = np.array([[-0.2, 0.3, 0.4], [d.lx + 0.5, d.ly + 1.0, -3.0]])
    clamped = np.clip(out, 0.0, [d.lx, d.ly, d.lz])
    np.testing.assert_allclose(dg.interpolate_velocity(pb, x, out), dg.interpolate_velocity(pb, x, clamped))


def test_tracking_moves_points_by_dt_times_velocity():
    pb = _problem(dt=0.02)
    v = np.array([0.3, -0.1, 0.7])
    x = _linear_velocity(pb, np.zeros((3, 3)), v)
    pts = np.array([[0.1, 0.2, 0.3], [0.55, 0.41, 0.9]])
    np.testing.assert_allclose(dg.track_points(pb, x, pts), pts + 0.02 * v, rtol=1e-14)
    # a rigid rotation about the box axis: one Euler step moves along the tangent
    A = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    x = _linear_velocity(pb, A, -A @ np.array([0.5, 0.4, 0.0]))
    p = np.array([[0.7, 0.4, 0.6]])
    assert dg.track_points(pb, x, p) == pytest.approx(np.array([[0.7, 0.4 + 0.02 * 0.2, 0.6]]), abs=1e-14)
