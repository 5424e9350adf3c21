"""Pins of the oracle's Allen-Cahn (Eq. PPV_AC) and B-transport (Eq. semiCGT) operators."""
import math

import numpy as np
import pytest

from oracle import ac, cgt, mobility
from oracle.fields import Problem, State
from tests.helpers import desc_small, rel, state_of
from workloads import node_coords


def _steady(x):
    return State(x.copy(), x.copy(), np.zeros_like(x))


def _tanh_residual(n):
    d = desc_small(n=(n, 2, 2), L=(1.0, 2.0 / n, 2.0 / n), dirichlet=False, n_fluid=1, n_solid=0,
                   eps=0.08)
    pb = Problem(d)
    X = node_coords(d)
    x = np.zeros((d.ncomp, d.nn))
    x[4] = np.tanh((X[0] - 0.5) / (math.sqrt(2.0) * d.eps))
    st = _steady(x)
    b = mobility.beta(pb, st, 0)
    r = ac.ac_residual(pb, st, 0, 1.0, b)
    # scale: the reaction term alone, node by node
    m = pb.mesh
    phi = m.val(x[4])
    scale = m.integrate(np.abs(phi ** 3 - phi), None)
    i = m.ijk()[0]
    inner = (i > 2) & (i < n - 2)
    return np.abs(r[inner]).max() / scale[inner].max(), b


def test_tanh_profile_is_discrete_equilibrium_at_second_order():
    """phi = tanh((x - 1/2)/(sqrt2 eps)) solves eps^2 phi'' = F'(phi) (Section 3, Eq.
    Allen-Cahn at rest): beta = 0 by symmetry and the discrete residual falls as h^2."""
    e1, b1 = _tanh_residual(40)
    e2, b2 = _tanh_residual(80)
    assert abs(b1) < 1e-12 and abs(b2) < 1e-12
    rate = math.log(e1 / e2, 2)
    assert 1.8 < rate < 2.3, rate


def test_residual_sum_identity_conserves_mass():
    """sum_a R_a = int (dphi^{n+alpha_m} + v.grad phi) + gamma (int F' - beta int sqrt F):
    the diffusion and SUPG terms carry grad N_a and sum to zero, and with beta from its
    definition the source integrates to zero, so at rest a converged solve keeps
    int phi (Section 2.2.1)."""
    d = desc_small(n=(3, 4, 3), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    st = state_of(d, 21)
    for i in range(2):
        b = mobility.beta(pb, st, i)
        r = ac.ac_residual(pb, st, i, 0.7, b)
        m = pb.mesh
        xa = pb.at_alpha(st)
        dphi = m.val(pb.at_alpha_m(st)[pb.phi_comp(i)])
        gphi = m.grad(xa[pb.phi_comp(i)])
        conv = sum(m.val(xa[j]) * gphi[..., j] for j in range(3))
        assert r.sum() == pytest.approx(m.integrate_scalar(dphi + conv), rel=1e-11, abs=1e-13)
        r0 = ac.ac_residual(pb, st, i, 0.7, 0.0)
        phi = m.val(xa[pb.phi_comp(i)])
        assert r0.sum() == pytest.approx(m.integrate_scalar(dphi + conv + 0.7 * (phi ** 3 - phi)), rel=1e-11)


def test_two_phase_antisymmetry():
    """phi_2 = -phi_1 is preserved: F' odd, beta odd, sqrt F, tau_phi and gamma even, so
    R(-phi) = -R(phi) and the Jacobians agree."""
    d = desc_small(n=(3, 3, 3), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    st = state_of(d, 4)
    for arr in (st.x, st.xn, st.xdn):
        arr[5] = -arr[4]
    g0, g1 = mobility.mobility(pb, st, 0), mobility.mobility(pb, st, 1)
    b0, b1 = mobility.beta(pb, st, 0), mobility.beta(pb, st, 1)
    assert g0 == pytest.approx(g1, rel=1e-14)
    assert b0 == pytest.approx(-b1, rel=1e-14)
    r0 = ac.ac_residual(pb, st, 0, g0, b0)
    r1 = ac.ac_residual(pb, st, 1, g1, b1)
    assert np.allclose(r0, -r1, rtol=1e-13, atol=1e-15)
    dphi = np.random.default_rng(0).normal(size=d.nn)
    assert np.allclose(ac.ac_jvp(pb, st, 0, g0, b0, dphi), ac.ac_jvp(pb, st, 1, g1, b1, dphi),
                       rtol=1e-13, atol=1e-15)


def test_ac_jvp_matches_central_differences():
    d = desc_small(n=(3, 2, 4), n_fluid=2, n_solid=1)
    pb = Problem(d)
    st = state_of(d, 8)
    i = 1
    dphi = np.random.default_rng(5).normal(size=d.nn)
    J = ac.ac_jvp(pb, st, i, 0.6, 0.2, dphi)
    h = 1e-6
    sp_, sm_ = State(st.x.copy(), st.xn, st.xdn), State(st.x.copy(), st.xn, st.xdn)
    sp_.x[4 + i] += h * dphi
    sm_.x[4 + i] -= h * dphi
    fd = (ac.ac_residual(pb, sp_, i, 0.6, 0.2, coef=st) - ac.ac_residual(pb, sm_, i, 0.6, 0.2, coef=st)) / (2 * h)
    assert rel(J, fd) < 1e-7


def test_ac_jvp_symmetric_at_rest():
    d = desc_small(n=(3, 3, 2), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    st = state_of(d, 12)
    st.x[0:3] = st.xn[0:3] = 0.0
    rng = np.random.default_rng(6)
    a, b = rng.normal(size=d.nn), rng.normal(size=d.nn)
    lhs = a @ ac.ac_jvp(pb, st, 0, 0.5, 0.1, b)
    rhs = b @ ac.ac_jvp(pb, st, 0, 0.5, 0.1, a)
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ------------------------------------------------------------------ B transport

def _linear_velocity(d, A, u0=(0.0, 0.0, 0.0)):
    X = node_coords(d)
    return np.asarray(A) @ X + np.asarray(u0)[:, None]


def test_rigid_motion_keeps_identity():
    """v = w x (x - c) + u0 (exact in Q1), B = I, dB = 0: Rb = 0 at every node."""
    d = desc_small(n=(3, 4, 3), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    w = np.array([0.3, -0.7, 1.1])
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    x = np.zeros((d.ncomp, d.nn))
    x[0:3] = _linear_velocity(d, W, (0.2, -0.1, 0.4))
    x[4] = -0.3
    x[5] = 0.3 + 0.5 * np.random.default_rng(0).uniform(-1, 1, d.nn)
    x[pb.b_comp(0, 0): pb.b_comp(0, 3)] = 1.0
    r = cgt.cgt_residual(pb, _steady(x), 0)
    assert np.abs(r).max() < 1e-15


def test_uniform_strain_rate_balances_stretching():
    """v = A x with a non-symmetric A, constant B, alpha = 1, dB/dt = A B + B A^T: the
    stretching terms grad v B + B grad v^T cancel the rate exactly (a transposed
    velocity gradient would not)."""
    d = desc_small(n=(3, 3, 3), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    A = np.array([[0.2, 0.5, -0.1], [-0.3, 0.1, 0.4], [0.6, -0.2, -0.3]])
    B = np.array([[1.2, 0.1, -0.05], [0.1, 0.9, 0.2], [-0.05, 0.2, 1.1]])
    rate = A @ B + B @ A.T
    x = np.zeros((d.ncomp, d.nn))
    x[0:3] = _linear_velocity(d, A)
    x[4], x[5] = -1.0, 1.0
    from oracle.fields import SYM
    xdn = np.zeros_like(x)
    for c, (k, l) in enumerate(SYM):
        x[pb.b_comp(0, c)] = B[k, l]
        xdn[pb.b_comp(0, c)] = rate[k, l] / (1.0 - pb.ga.alpha_m)  # dB^{n+alpha_m} when x^{n+1} = x^n
    st = State(x, x.copy(), xdn)
    r = cgt.cgt_residual(pb, st, 0)
    assert np.abs(r).max() < 1e-14
    # and the transposed variant does not vanish
    wrong = A.T @ B + B @ A
    for c, (k, l) in enumerate(SYM):
        xdn[pb.b_comp(0, c)] = wrong[k, l] / (1.0 - pb.ga.alpha_m)
    assert np.abs(cgt.cgt_residual(pb, State(x, x.copy(), xdn), 0)).max() > 1e-4


def test_recovery_term_closed_form():
    """alpha^s = 0 (phi^s = -1), v = 0, B = I + D: R_a = D int N_a (lumped mass)."""
    d = desc_small(n=(3, 2, 3), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    x = np.zeros((d.ncomp, d.nn))
    x[4], x[5] = 1.0, -1.0
    D = [0.1, -0.2, 0.05, 0.3, -0.1, 0.02]
    for c in range(6):
        x[pb.b_comp(0, c)] = (1.0 if c < 3 else 0.0) + D[c]
    r = cgt.cgt_residual(pb, _steady(x), 0)
    lump = pb.mesh.integrate(np.ones((pb.mesh.ne, 8)))
    for c in range(6):
        assert np.allclose(r[c], D[c] * lump, rtol=1e-13, atol=1e-17)


def test_cgt_jvp_is_exact_derivative_of_linear_residual():
    d = desc_small(n=(2, 3, 3), n_fluid=1, n_solid=2)
    pb = Problem(d)
    st = state_of(d, 14)
    dB = np.random.default_rng(7).normal(size=(6, d.nn))
    for s in range(2):
        sp_ = State(st.x.copy(), st.xn, st.xdn)
        for c in range(6):
            sp_.x[pb.b_comp(s, c)] += dB[c]
        fd = cgt.cgt_residual(pb, sp_, s, coef=st) - cgt.cgt_residual(pb, st, s)
        assert rel(cgt.cgt_jvp(pb, st, s, dB), fd) < 1e-12
