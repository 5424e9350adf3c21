"""Unified momentum/continuity residual and Jacobian-vector product (oracle).

Test infrastructure only (see oracle/__init__.py).

Eq. (PG_NS), Section 2.1.2, with
  rho = sum_i alpha^i rho^i, mu = sum_i alpha^i mu^i, alpha^i = (1+phi^i)/2  (Section 2.1.1)
  sigma = -p I + mu (grad v + grad v^T) + sum_s alpha^s mu_L^s (B^s - I)
          (Newtonian stress, Section 2.2; Neo-Hookean stress, Section 2.3.1; the
          pressure is not weighted, only the viscous and elastic parts are blended)
  body force b = rho g
  R_m = rho (dv/dt + v.grad v) + grad p - rho g    (strong momentum residual; the
          divergence of the stress is dropped: zero for the paper's linear elements)
  R_c = div v
  tau_m = ((2/dt)^2 + v.G v + C_I (mu/rho)^2 G:G)^(-1/2),  tau_c = 1/(tr(G) tau_m)

For node a and component k the momentum residual is
  int rho (dv_k + v_j d_j v_k - g_k) N_a
  + int sigma_kj d_j N_a
  + int tau_m (v_j d_j N_a) R_m,k            (SUPG: (tau_m/rho)(rho v.grad psi).R_m)
  + int tau_c rho R_c d_k N_a                (LSIC)
and the continuity residual is
  int N_a R_c + int (tau_m/rho) d_j N_a R_m,j  (PSPG).
Velocities, phases and B are at n+alpha, dv/dt at n+alpha_m, p at n+1.
Dirichlet rows return x - x_D.

The Jacobian-vector product differentiates this in (v^{n+1}, p^{n+1}) with tau_m,
tau_c, phi and B frozen, and (flag elastic_aug) adds the solid-stress linearization of
Section 2.4 / Appendix B:
  sum_s int alpha^s mu_L^s dB^s_kj d_j N_a,
  dB^s = (alpha vs dt / alpha_m) ( -(dv.grad) B^s + grad(dv) B^s + B^s grad(dv)^T ),
with dv the increment of v^{n+alpha}.  Dirichlet rows are the identity.
"""
from __future__ import annotations

import numpy as np

from .bc import dirichlet
from .fields import Problem, State


def _tau(pb: Problem, coef: State):
    """tau_m, tau_c at quadrature points from the coefficient state."""
    xa = pb.at_alpha(coef)
    vq, _ = pb.velocity(xa)
    rho, mu, _ = pb.materials(xa)
    d = pb.desc
    nu = mu / rho
    tau_m = (4.0 / d.dt ** 2 + pb.vGv(vq) + d.c_i * nu ** 2 * pb.GG) ** -0.5
    tau_c = 1.0 / (pb.trG * tau_m)
    return tau_m, tau_c


def _elastic_stress(pb: Problem, xa, alphas):
    """sum_s alpha^s mu_L^s (B^s - I) -> (3,3,ne,8)."""
    E = 0.0
    for s, ph_i in enumerate(pb.solids):
        B, _ = pb.b_tensor(xa, s, with_grad=False)
        Bm = B.copy()
        for k in range(3):
            Bm[k, k] -= 1.0
        E = E + alphas[ph_i] * pb.desc.phases[ph_i].mu_L * Bm
    return E


def _strong_momentum(pb: Problem, st: State):
    """R_m (3, ne, 8) and the pieces it is built from."""
    m = pb.mesh
    xa = pb.at_alpha(st)
    xd = pb.at_alpha_m(st)
    vq, gvq = pb.velocity(xa)
    rho, mu, alphas = pb.materials(xa)
    gp = m.grad(st.x[3])
    g = pb.desc.gravity
    acc = np.stack([m.val(xd[k]) + sum(vq[j] * gvq[k][..., j] for j in range(3)) for k in range(3)])
    Rm = np.stack([rho * acc[k] + gp[..., k] - rho * g[k] for k in range(3)])
    return xa, vq, gvq, rho, mu, alphas, acc, Rm


def ns_residual(pb: Problem, st: State, coef: State | None = None) -> np.ndarray:
    """(4, nn): momentum components 0..2 and continuity 3."""
    coef = st if coef is None else coef
    m = pb.mesh
    tau_m, tau_c = _tau(pb, coef)
    xa, vq, gvq, rho, mu, alphas, acc, Rm = _strong_momentum(pb, st)
    pq = m.val(st.x[3])
    Rc = gvq[0][..., 0] + gvq[1][..., 1] + gvq[2][..., 2]
    E = _elastic_stress(pb, xa, alphas)
    g = pb.desc.gravity
    out = np.empty((4, m.nn))
    for k in range(3):
        f = rho * (acc[k] - g[k])
        gk = np.empty(f.shape + (3,))
        for j in range(3):
            sig = mu * (gvq[k][..., j] + gvq[j][..., k]) + (E[k, j] if np.ndim(E) else 0.0)
            if j == k:
                sig = sig - pq + tau_c * rho * Rc
            gk[..., j] = sig + tau_m * vq[j] * Rm[k]
        out[k] = m.integrate(f, gk)
    gc = np.stack([tau_m / rho * Rm[j] for j in range(3)], axis=-1)
    out[3] = m.integrate(Rc, gc)
    vmask, vD, pmask = dirichlet(pb.desc)
    for k in range(3):
        out[k, vmask] = st.x[k, vmask] - vD[k, vmask]
    out[3, pmask] = st.x[3, pmask]
    return out


def ns_jvp(pb: Problem, st: State, dx: np.ndarray, elastic_aug: bool = True) -> np.ndarray:
    """(4, nn) = J_NS(st) dx with dx (4, nn) = (dv, dp) increments of (v^{n+1}, p^{n+1})."""
    m = pb.mesh
    ga = pb.ga
    tau_m, tau_c = _tau(pb, st)
    xa, vq, gvq, rho, mu, alphas, acc, Rm = _strong_momentum(pb, st)
    # increments of v^{n+alpha}, dv/dt^{n+alpha_m} and p^{n+1}
    dva = np.stack([ga.alpha * m.val(dx[k]) for k in range(3)])
    gdva = np.stack([ga.alpha * m.grad(dx[k]) for k in range(3)])
    ddot = np.stack([ga.c_mass * m.val(dx[k]) for k in range(3)])
    dpq = m.val(dx[3])
    gdp = m.grad(dx[3])
    dacc = np.stack([ddot[k] + sum(dva[j] * gvq[k][..., j] + vq[j] * gdva[k][..., j] for j in range(3))
                     for k in range(3)])
    dRm = np.stack([rho * dacc[k] + gdp[..., k] for k in range(3)])
    dRc = gdva[0][..., 0] + gdva[1][..., 1] + gdva[2][..., 2]
    # elastic linearization (Section 2.4): dB = c ( -(dv.grad)B + grad(dv) B + B grad(dv)^T )
    dE = None
    if elastic_aug and pb.ns > 0:
        c = ga.c_elastic
        dE = 0.0
        for s, ph_i in enumerate(pb.solids):
            B, gB = pb.b_tensor(xa, s, with_grad=True)
            dB = np.empty_like(B)
            for k in range(3):
                for l in range(3):
                    t = -sum(dva[mm] * gB[k, l][..., mm] for mm in range(3))
                    t = t + sum(gdva[k][..., mm] * B[mm, l] for mm in range(3))
                    t = t + sum(B[k, mm] * gdva[l][..., mm] for mm in range(3))
                    dB[k, l] = c * t
            dE = dE + alphas[ph_i] * pb.desc.phases[ph_i].mu_L * dB
    out = np.empty((4, m.nn))
    for k in range(3):
        f = rho * dacc[k]
        gk = np.empty(f.shape + (3,))
        for j in range(3):
            sig = mu * (gdva[k][..., j] + gdva[j][..., k])
            if dE is not None:
                sig = sig + dE[k, j]
            if j == k:
                sig = sig - dpq + tau_c * rho * dRc
            gk[..., j] = sig + tau_m * dva[j] * Rm[k] + tau_m * vq[j] * dRm[k]
        out[k] = m.integrate(f, gk)
    gc = np.stack([tau_m / rho * dRm[j] for j in range(3)], axis=-1)
    out[3] = m.integrate(dRc, gc)
    vmask, _, pmask = dirichlet(pb.desc)
    for k in range(3):
        out[k, vmask] = dx[k, vmask]
    out[3, pmask] = dx[3, pmask]
    return out


def elastic_tilde_stress_residual(pb: Problem, st: State, v_np1: np.ndarray) -> np.ndarray:
    """(3, nn): sum_s int alpha^s mu_L^s Btilde^s(v) : grad N_a, the map whose
    derivative in v^{n+1} the elastic augmentation is (Section 2.4, Eq. Bext with the
    evolution equation substituted; B on the right-hand side frozen at st):
      Btilde(v) = B^n + alpha dt ((1 - vs/alpha_m) dB^n + (vs/alpha_m) F(v)),
      F(v) = -(v.grad) B + grad v B + B grad v^T,  v = v^{n+alpha}(v^{n+1}).
    Used only by tests of the augmentation."""
    m = pb.mesh
    ga = pb.ga
    xa = pb.at_alpha(st)
    _, _, alphas = pb.materials(xa)
    va = ga.at_alpha(v_np1, st.xn[0:3])
    vq = np.stack([m.val(va[k]) for k in range(3)])
    gvq = np.stack([m.grad(va[k]) for k in range(3)])
    out = np.zeros((3, m.nn))
    for s, ph_i in enumerate(pb.solids):
        B, gB = pb.b_tensor(xa, s, with_grad=True)
        comp_n = [m.val(st.xn[pb.b_comp(s, c)]) for c in range(6)]
        compd_n = [m.val(st.xdn[pb.b_comp(s, c)]) for c in range(6)]
        from .fields import SYM_INDEX
        coef = alphas[ph_i] * pb.desc.phases[ph_i].mu_L
        for k in range(3):
            gk = np.zeros(vq[0].shape + (3,))
            for l in range(3):
                F = -sum(vq[mm] * gB[k, l][..., mm] for mm in range(3))
                F = F + sum(gvq[k][..., mm] * B[mm, l] for mm in range(3))
                F = F + sum(B[k, mm] * gvq[l][..., mm] for mm in range(3))
                idx = SYM_INDEX[k, l]
                Bt = comp_n[idx] + ga.alpha * ga.dt * ((1.0 - ga.vs / ga.alpha_m) * compd_n[idx]
                                                       + (ga.vs / ga.alpha_m) * F)
                gk[..., l] = coef * Bt
            out[k] += m.integrate(None, gk)
    return out
