"""Pins of the oracle's momentum/continuity residual and JVP (Eq. PG_NS, Section 2.4)."""
import numpy as np
import pytest

from oracle import ns
from oracle.bc import dirichlet
from oracle.fields import Problem, State
from tests.helpers import desc_small, rel, state_of


def _interior(pb):
    i, j, k = pb.mesh.ijk()
    d = pb.desc
    return (i > 0) & (i < d.nx) & (j > 0) & (j < d.ny) & (k > 0) & (k < d.nz)


def _steady(pb, x):
    return State(x.copy(), x.copy(), np.zeros_like(x))


def test_couette_patch_interior_residual_vanishes():
    """v = (z, 0, 0): (v.grad)v = 0, div v = 0, constant viscous and elastic stress,
    constant p, steady: every interior momentum and continuity residual is zero."""
    d = desc_small(n=(4, 3, 5))
    pb = Problem(d)
    i, j, k = pb.mesh.ijk()
    z = k * pb.mesh.h[2]
    x = np.zeros((d.ncomp, d.nn))
    x[0] = z
    x[3] = 0.37
    x[4] = 0.2   # phase indicators constant
    x[5] = -0.4
    Bc = [1.1, 0.9, 1.05, 0.03, -0.02, 0.01]
    for c in range(6):
        x[pb.b_comp(0, c)] = Bc[c]
    r = ns.ns_residual(pb, _steady(pb, x))
    inner = _interior(pb)
    assert np.abs(r[:, inner]).max() < 1e-14


def test_hydrostatic_balance():
    """p = rho g.x with uniform rho balances gravity: interior residual zero."""
    d = desc_small(n=(3, 4, 3), gravity=(0.0, 0.0, -9.81), n_solid=0)
    pb = Problem(d)
    i, j, k = pb.mesh.ijk()
    x = np.zeros((d.ncomp, d.nn))
    x[4] = 1.0  # single phase, alpha = 1 -> rho = rho_0
    rho = d.phases[0].rho
    x[3] = rho * (-9.81) * (k * pb.mesh.h[2])
    r = ns.ns_residual(pb, _steady(pb, x))
    assert np.abs(r[:, _interior(pb)]).max() < 1e-12


def test_mass_term_closed_form():
    """v = 0, uniform dv/dt^{n+alpha_m} = a: interior momentum residual = rho a_k h^3."""
    d = desc_small(n=(4, 4, 4), n_solid=0)
    pb = Problem(d)
    x = np.zeros((d.ncomp, d.nn))
    x[4] = 1.0
    a = np.array([0.3, -1.2, 0.5])
    xdn = np.zeros_like(x)
    xdn[0:3] = a[:, None]  # with x^{n+1} = x^n: dv^{n+alpha_m} = (1 - alpha_m) xdot^n ...
    st = State(x.copy(), x.copy(), xdn)
    xd = pb.at_alpha_m(st)
    r = ns.ns_residual(pb, st)
    h3 = np.prod(pb.mesh.h)
    inner = _interior(pb)
    for kk in range(3):
        assert np.allclose(r[kk, inner], d.phases[0].rho * xd[kk, inner] * h3, rtol=1e-13)


def test_dirichlet_rows():
    d = desc_small(n=(3, 3, 3))
    pb = Problem(d)
    st = state_of(d, 3)
    r = ns.ns_residual(pb, st)
    vmask, vD, pmask = dirichlet(d)
    assert np.array_equal(r[0:3, vmask], st.x[0:3, vmask] - vD[:, vmask])
    assert np.array_equal(r[3, pmask], st.x[3, pmask])
    # lid (z = 1) wins on its edges
    i, j, k = pb.mesh.ijk()
    assert np.all(vD[0, k == d.nz] == 1.0)
    assert np.all(vD[0, (k < d.nz) & vmask] == 0.0)


@pytest.mark.parametrize("rho_inf", [0.0, 0.5])
def test_jvp_matches_central_differences(rho_inf):
    """J dx = d/dh R(x + h dx) with tau and the coefficient state frozen (no elastic
    augmentation, which is not a derivative of the residual)."""
    d = desc_small(n=(3, 2, 3), gravity=(0.0, -1.0, -9.81), n_fluid=2, n_solid=2, rho_inf=rho_inf)
    pb = Problem(d)
    st = state_of(d, 5)
    dx = np.random.default_rng(9).normal(size=(4, d.nn))
    Jdx = ns.ns_jvp(pb, st, dx, elastic_aug=False)
    h = 1e-5
    sp, sm = State(st.x.copy(), st.xn, st.xdn), State(st.x.copy(), st.xn, st.xdn)
    sp.x[0:4] += h * dx
    sm.x[0:4] -= h * dx
    fd = (ns.ns_residual(pb, sp, coef=st) - ns.ns_residual(pb, sm, coef=st)) / (2 * h)
    assert rel(Jdx, fd) < 1e-7


def test_elastic_augmentation_is_derivative_of_btilde_stress():
    """The augmentation equals the derivative in v^{n+1} of
    sum_s int alpha^s mu_L^s Btilde^s(v) : grad N_a (Section 2.4), which is linear."""
    d = desc_small(n=(3, 3, 2), n_fluid=1, n_solid=2)
    pb = Problem(d)
    st = state_of(d, 11)
    dx = np.random.default_rng(2).normal(size=(4, d.nn))
    dx[3] = 0.0
    aug = ns.ns_jvp(pb, st, dx, True) - ns.ns_jvp(pb, st, dx, False)
    vmask, _, _ = dirichlet(d)
    base = ns.elastic_tilde_stress_residual(pb, st, st.x[0:3])
    pert = ns.elastic_tilde_stress_residual(pb, st, st.x[0:3] + dx[0:3])
    fd = pert - base
    free = ~vmask
    assert rel(aug[0:3, free], fd[:, free]) < 1e-11
    assert np.all(aug[3] == 0.0)


def test_appendix_b_component_form_2d_slice():
    """The 3D augmentation restricted to a field with v_z = 0, no z-variation and
    B13 = B23 = 0 reproduces Appendix B's 2D component form of
    mu_L d(N,x B11 + N,y B12)/d v_x (its gamma is the paper's varsigma)."""
    d = desc_small(n=(3, 3, 1), n_fluid=1, n_solid=1, dirichlet=False)
    pb = Problem(d)
    m = pb.mesh
    rng = np.random.default_rng(4)
    i, j, k = m.ijk()
    X, Y = i * m.h[0], j * m.h[1]
    x = np.zeros((d.ncomp, d.nn))
    x[4], x[5] = -1.0, 1.0  # solid alpha = 1
    B11 = 1.0 + 0.1 * X + 0.05 * Y
    B22 = 1.0 - 0.07 * X + 0.02 * Y
    B12 = 0.03 + 0.04 * X - 0.06 * Y
    x[pb.b_comp(0, 0)], x[pb.b_comp(0, 1)], x[pb.b_comp(0, 2)] = B11, B22, 1.0
    x[pb.b_comp(0, 3)] = B12
    st = State(x, x.copy(), np.zeros_like(x))
    # trial: v_x = N_b at one node column (no z variation -> both z-nodes)
    b = (i == 1) & (j == 2)
    dx = np.zeros((4, d.nn))
    dx[0, b] = 1.0
    aug = ns.ns_jvp(pb, st, dx, True) - ns.ns_jvp(pb, st, dx, False)
    # Appendix B integrand for test N_a (row x), trial N_b in v_x, 2D, c = dt alpha vs / alpha_m
    ga = pb.ga
    c = ga.dt * ga.alpha * ga.vs / ga.alpha_m
    muL = d.phases[1].mu_L
    Nb = m.val(dx[0])
    gNb = m.grad(dx[0])
    gq = lambda u: m.grad(u)
    vq = lambda u: m.val(u)
    B11q, B12q, B22q = vq(B11), vq(B12), vq(B22)
    gB11, gB12 = gq(B11), gq(B12)
    # per test function: N_a,x * c(-N dB11/dx + 2 N,x B11 + 2 N,y B12) + N_a,y * c(-N dB12/dx + N,x B12 + N,y B22)
    gx = c * (-Nb * gB11[..., 0] + 2 * gNb[..., 0] * B11q + 2 * gNb[..., 1] * B12q)
    gy = c * (-Nb * gB12[..., 0] + gNb[..., 0] * B12q + gNb[..., 1] * B22q)
    g = np.stack([gx, gy, np.zeros_like(gx)], axis=-1) * muL
    expect = m.integrate(None, g)
    # the 3D form carries alpha^{n+alpha} = 1 in the solid and an alpha from d v^{n+alpha}/d v^{n+1}
    assert np.allclose(aug[0], ga.alpha * expect, rtol=1e-12, atol=1e-15)
    _ = rng


def test_jvp_symmetric_blocks_at_rest():
    """At v = 0, dv/dt = 0, p = 0, g = 0 and natural boundaries, the velocity-velocity
    block (mass + viscous + LSIC) and the pressure-pressure block (PSPG) are symmetric."""
    d = desc_small(n=(3, 3, 2), dirichlet=False, n_solid=1)
    pb = Problem(d)
    st = state_of(d, 7)
    st.x[0:4] = 0.0
    st.xn[0:4] = 0.0
    st.xdn[0:4] = 0.0
    rng = np.random.default_rng(3)
    a = rng.normal(size=(4, d.nn))
    b = rng.normal(size=(4, d.nn))
    au, bu = a.copy(), b.copy()
    au[3] = bu[3] = 0.0
    lhs = np.sum(au[0:3] * ns.ns_jvp(pb, st, bu, False)[0:3])
    rhs = np.sum(bu[0:3] * ns.ns_jvp(pb, st, au, False)[0:3])
    assert lhs == pytest.approx(rhs, rel=1e-12)
    ap, bp = np.zeros_like(a), np.zeros_like(b)
    ap[3], bp[3] = a[3], b[3]
    lhs = np.sum(ap[3] * ns.ns_jvp(pb, st, bp, False)[3])
    rhs = np.sum(bp[3] * ns.ns_jvp(pb, st, ap, False)[3])
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_tau_closed_form_uniform():
    """tau_m for v = 0 and one phase: (4/dt^2 + C_I (mu/rho)^2 48/h^4)^(-1/2)."""
    d = desc_small(n=(2, 2, 2), n_solid=0)
    pb = Problem(d)
    x = np.zeros((d.ncomp, d.nn))
    x[4] = 1.0
    tm, tc = ns._tau(pb, _steady(pb, x))
    h = pb.mesh.h[0]
    ph = d.phases[0]
    expect = (4.0 / d.dt ** 2 + d.c_i * (ph.mu / ph.rho) ** 2 * 48.0 / h ** 4) ** -0.5
    assert np.allclose(tm, expect, rtol=1e-14)
    assert np.allclose(tc, 1.0 / (12.0 / h ** 2 * expect), rtol=1e-14)
