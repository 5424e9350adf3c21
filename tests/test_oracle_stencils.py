"""Pins of the oracle's linearized operators against textbook Q1 matrices.

At a uniform state (constant velocity U, constant phase indicators, zero strong
momentum residual) every coefficient of the stabilized forms is constant, and each
term of the Jacobians is a product of the 1D Q1 matrices
    M1[a,b] = int N_a N_b,  K1[a,b] = int N_a' N_b',  C1[a,b] = int N_a N_b'
(tridiagonal, closed form), combined by Kronecker products in z (x) y (x) x order.
This pins the signs and scalings of the Galerkin, SUPG, PSPG and LSIC terms of
Eq. PG_NS, of the Allen-Cahn form (Eq. PPV_AC) and of the B transport (Eq. semiCGT).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ac, cgt, ns
from oracle.fields import Problem, State
from tests.helpers import desc_small


def _m1(n, h):
    d = np.full(n + 1, 2 * h / 3)
    d[0] = d[-1] = h / 3
    return sp.diags([np.full(n, h / 6), d, np.full(n, h / 6)], [-1, 0, 1])


def _k1(n, h):
    d = np.full(n + 1, 2 / h)
    d[0] = d[-1] = 1 / h
    return sp.diags([np.full(n, -1 / h), d, np.full(n, -1 / h)], [-1, 0, 1])


def _c1(n, h):
    d = np.zeros(n + 1)
    d[0], d[-1] = -0.5, 0.5
    return sp.diags([np.full(n, -0.5), d, np.full(n, 0.5)], [-1, 0, 1])


class Kron:
    def __init__(self, desc):
        n = (desc.nx, desc.ny, desc.nz)
        h = desc.h
        self.M = [_m1(n[d], h[d]) for d in range(3)]
        self.K = [_k1(n[d], h[d]) for d in range(3)]
        self.C = [_c1(n[d], h[d]) for d in range(3)]

    def _k(self, mats):
        return sp.kron(mats[2], sp.kron(mats[1], mats[0])).tocsr()

    def mass(self):
        return self._k(self.M)

    def conv(self, j):
        """int N_a d_j N_b."""
        m = list(self.M)
        m[j] = self.C[j]
        return self._k(m)

    def grad_grad(self, i, j):
        """int d_i N_a d_j N_b."""
        m = list(self.M)
        if i == j:
            m[i] = self.K[i]
        else:
            m[i] = self.C[i].T
            m[j] = self.C[j]
        return self._k(m)


def _uniform_state(d, U, phis, extra=None):
    x = np.zeros((d.ncomp, d.nn))
    x[0:3] = np.asarray(U)[:, None]
    for i, c in enumerate(phis):
        x[4 + i] = c
    base = 4 + d.n_phase
    for s in range(d.n_solid):
        x[base + 6 * s: base + 6 * s + 3] = 1.0
    if extra is not None:
        extra(x)
    return State(x, x.copy(), np.zeros_like(x))


@pytest.mark.parametrize("U", [(0.0, 0.0, 0.0), (0.7, -0.3, 1.1)])
def test_ns_jvp_equals_kronecker_operator(U):
    d = desc_small(n=(3, 4, 2), L=(1.0, 1.3, 0.6), dirichlet=False, n_fluid=1, n_solid=0)
    pb = Problem(d)
    ga = pb.ga
    st = _uniform_state(d, U, [1.0])
    U = np.asarray(U)
    ph = d.phases[0]
    rho, mu = ph.rho, ph.mu
    tau_m = (4 / d.dt ** 2 + (pb.Gd * U ** 2).sum() + d.c_i * (mu / rho) ** 2 * pb.GG) ** -0.5
    tau_c = 1 / (pb.trG * tau_m)
    kr = Kron(d)
    M = kr.mass()
    C = [kr.conv(j) for j in range(3)]
    E = [[kr.grad_grad(i, j) for j in range(3)] for i in range(3)]
    a, cm = ga.alpha, ga.c_mass
    rng = np.random.default_rng(0)
    dx = rng.normal(size=(4, d.nn))
    dv, dp = dx[0:3], dx[3]
    expect = np.zeros((4, d.nn))
    Ugrad = sum(U[j] * C[j] for j in range(3))
    UgradT = sum(U[i] * C[i].T for i in range(3))
    UU = sum(U[i] * U[j] * E[i][j] for i in range(3) for j in range(3))
    for k in range(3):
        r = rho * cm * (M @ dv[k]) + rho * a * (Ugrad @ dv[k])
        r += a * mu * sum(E[j][j] @ dv[k] for j in range(3))
        r += a * mu * sum(E[j][k] @ dv[j] for j in range(3))
        r -= C[k].T @ dp
        r += tau_c * rho * a * sum(E[k][j] @ dv[j] for j in range(3))
        r += tau_m * (rho * cm * (UgradT @ dv[k]) + rho * a * (UU @ dv[k])
                      + sum(U[i] * (E[i][k] @ dp) for i in range(3)))
        expect[k] = r
    c = a * sum(C[j] @ dv[j] for j in range(3))
    c += tau_m / rho * sum(E[j][j] @ dp + rho * cm * (C[j].T @ dv[j])
                           + rho * a * sum(U[i] * (E[j][i] @ dv[j]) for i in range(3))
                           for j in range(3))
    expect[3] = c
    got = ns.ns_jvp(pb, st, dx, elastic_aug=True)
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


@pytest.mark.parametrize("U,c", [((0.0, 0.0, 0.0), 0.3), ((0.4, 0.9, -0.6), -0.45), ((0.1, 0.0, 0.2), 1.2)])
def test_ac_jvp_equals_kronecker_operator(U, c):
    d = desc_small(n=(4, 3, 3), L=(1.0, 0.8, 0.9), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    ga = pb.ga
    gamma, beta = 0.8, 0.35
    st = _uniform_state(d, U, [c, -c])
    U = np.asarray(U)
    eps2 = d.eps ** 2
    Fpp = 3 * c * c - 1
    dsF = c * np.sign(c * c - 1)
    rp = Fpp - beta * dsF
    tau = (4 / d.dt ** 2 + (pb.Gd * U ** 2).sum() + 9 * (gamma * eps2) ** 2 * pb.GG + (gamma * Fpp) ** 2) ** -0.5
    kr = Kron(d)
    M = kr.mass()
    C = [kr.conv(j) for j in range(3)]
    E = [[kr.grad_grad(i, j) for j in range(3)] for i in range(3)]
    a, cm = ga.alpha, ga.c_mass
    Ugrad = sum(U[j] * C[j] for j in range(3))
    UgradT = sum(U[i] * C[i].T for i in range(3))
    UU = sum(U[i] * U[j] * E[i][j] for i in range(3) for j in range(3))
    J = (cm + gamma * a * rp) * M + a * Ugrad + gamma * eps2 * a * sum(E[j][j] for j in range(3))
    J = J + tau * ((cm + gamma * a * rp) * UgradT + a * UU)
    dphi = np.random.default_rng(1).normal(size=d.nn)
    got = ac.ac_jvp(pb, st, 0, gamma, beta, dphi)
    expect = J @ dphi
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


@pytest.mark.parametrize("U,c", [((0.0, 0.0, 0.0), 0.5), ((0.3, -0.8, 0.5), -0.2)])
def test_cgt_jvp_equals_kronecker_operator(U, c):
    d = desc_small(n=(3, 3, 4), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    ga = pb.ga
    st = _uniform_state(d, U, [-c, c])
    U = np.asarray(U)
    al = (1 + c) / 2
    tau = (4 / d.dt ** 2 + (pb.Gd * U ** 2).sum()) ** -0.5
    kr = Kron(d)
    M = kr.mass()
    C = [kr.conv(j) for j in range(3)]
    E = [[kr.grad_grad(i, j) for j in range(3)] for i in range(3)]
    a, cm = ga.alpha, ga.c_mass
    Ugrad = sum(U[j] * C[j] for j in range(3))
    UgradT = sum(U[i] * C[i].T for i in range(3))
    UU = sum(U[i] * U[j] * E[i][j] for i in range(3) for j in range(3))
    react = al * cm + (1 - al) * a
    J = react * M + al * a * Ugrad + tau * (react * UgradT + al * a * UU)
    dB = np.random.default_rng(2).normal(size=(6, d.nn))
    got = cgt.cgt_jvp(pb, st, 0, dB)
    expect = np.stack([J @ dB[k] for k in range(6)])
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


def test_pspg_block_is_scaled_q1_laplacian_stencil():
    """Interior row of the pressure-pressure block at rest: (tau_m/rho) times the Q1
    Laplacian stencil h/3 [8 centre, 0 faces, -1/2 edges, -1/4 corners]."""
    d = desc_small(n=(4, 4, 4), dirichlet=False, n_fluid=1, n_solid=0)
    pb = Problem(d)
    st = _uniform_state(d, (0.0, 0.0, 0.0), [1.0])
    centre = 2 + 5 * (2 + 5 * 2)
    dx = np.zeros((4, d.nn))
    dx[3, centre] = 1.0
    y = ns.ns_jvp(pb, st, dx)[3]
    ph = d.phases[0]
    h = pb.mesh.h[0]
    tau_m = (4 / d.dt ** 2 + d.c_i * (ph.mu / ph.rho) ** 2 * pb.GG) ** -0.5
    i, j, k = pb.mesh.ijk()
    off = np.abs(i - 2) + np.abs(j - 2) + np.abs(k - 2)
    near = (np.abs(i - 2) <= 1) & (np.abs(j - 2) <= 1) & (np.abs(k - 2) <= 1)
    stencil = {0: 8.0, 1: 0.0, 2: -0.5, 3: -0.25}
    for n in np.nonzero(near)[0]:
        assert y[n] == pytest.approx(tau_m / ph.rho * h / 3 * stencil[int(off[n])], rel=1e-12, abs=1e-16)
    assert np.all(y[~near] == 0.0)
