"""Allen-Cahn residual and Jacobian-vector product of one phase indicator (oracle).

Test infrastructure only (see oracle/__init__.py).

Strong form (Eq. Allen-Cahn, Section 2.2.1):
  dphi/dt + v.grad phi = -gamma (F'(phi) - eps^2 lap phi - beta sqrt(F(phi))),
  F = (phi^2 - 1)^2 / 4,  F' = phi^3 - phi,  sqrt(F) = |phi^2 - 1| / 2.
Variational form (Eq. PPV_AC, Section 2.2.3) with the diffusion, reaction and source
coefficients read as their plain Galerkin values (k = eps^2 under gamma; reaction
and source together gamma (F'(phi) - beta sqrt F)):
  int N_a (dphi + v.grad phi) + gamma [eps^2 grad N_a . grad phi
                                       + N_a (F'(phi) - beta sqrt F(phi))]
  + int tau_phi (v.grad N_a) R_phi,
  R_phi = dphi + v.grad phi + gamma (F'(phi) - beta sqrt F(phi))   (the eps^2 lap phi
          term is dropped from the element residual: zero for linear elements),
  tau_phi = ((2/dt)^2 + v.G v + 9 khat^2 G:G + shat^2)^(-1/2),
  khat = gamma eps^2, shat = gamma F''(phi) = gamma (3 phi^2 - 1).
phi at n+alpha, dphi at n+alpha_m, v at n+alpha (frozen in this block).  gamma and
beta are frozen scalars of the block.  No Dirichlet rows.

The Jacobian-vector product differentiates in phi^{n+1} with gamma, beta and
tau_phi frozen; d sqrt(F)/d phi = phi sign(phi^2 - 1), taken as 0 at |phi| = 1.
"""
from __future__ import annotations

import numpy as np

from .fields import Problem, State


def _coeffs(pb: Problem, coef: State, i: int, gamma: float):
    m = pb.mesh
    xa = pb.at_alpha(coef)
    vq, _ = pb.velocity(xa)
    phi = m.val(xa[pb.phi_comp(i)])
    d = pb.desc
    khat = gamma * d.eps ** 2
    shat = gamma * (3.0 * phi ** 2 - 1.0)
    tau = (4.0 / d.dt ** 2 + pb.vGv(vq) + 9.0 * khat ** 2 * pb.GG + shat ** 2) ** -0.5
    return vq, tau


def ac_residual(pb: Problem, st: State, i: int, gamma: float, beta: float,
                coef: State | None = None) -> np.ndarray:
    coef = st if coef is None else coef
    m = pb.mesh
    vq, tau = _coeffs(pb, coef, i, gamma)
    xa = pb.at_alpha(st)
    xd = pb.at_alpha_m(st)
    c = pb.phi_comp(i)
    phi = m.val(xa[c])
    gphi = m.grad(xa[c])
    dphi = m.val(xd[c])
    Fp = phi ** 3 - phi
    sF = 0.5 * np.abs(phi ** 2 - 1.0)
    conv = sum(vq[j] * gphi[..., j] for j in range(3))
    R = dphi + conv + gamma * (Fp - beta * sF)
    eps2 = pb.desc.eps ** 2
    g = np.stack([gamma * eps2 * gphi[..., j] + tau * vq[j] * R for j in range(3)], axis=-1)
    return m.integrate(R, g)


def ac_jvp(pb: Problem, st: State, i: int, gamma: float, beta: float, dphi_np1: np.ndarray) -> np.ndarray:
    m = pb.mesh
    ga = pb.ga
    vq, tau = _coeffs(pb, st, i, gamma)
    xa = pb.at_alpha(st)
    phi = m.val(xa[pb.phi_comp(i)])
    dpa = ga.alpha * m.val(dphi_np1)
    gdpa = ga.alpha * m.grad(dphi_np1)
    ddot = ga.c_mass * m.val(dphi_np1)
    Fpp = 3.0 * phi ** 2 - 1.0
    dsF = phi * np.sign(phi ** 2 - 1.0)
    dR = ddot + sum(vq[j] * gdpa[..., j] for j in range(3)) + gamma * (Fpp - beta * dsF) * dpa
    eps2 = pb.desc.eps ** 2
    g = np.stack([gamma * eps2 * gdpa[..., j] + tau * vq[j] * dR for j in range(3)], axis=-1)
    return m.integrate(dR, g)
