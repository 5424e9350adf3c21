"""Time-dependent mobility gamma and the Lagrange multiplier beta (oracle).

Test infrastructure only (see oracle/__init__.py).

gamma (Section 2.2.2, discrete mobility model):
  q = (grad phi)^T grad v (grad phi) / |grad phi|^2 at quadrature points,
      (grad v)_jk = d v_j / d x_k  (Appendix B component form); q = 0 where
      |grad phi|^2 < 1e-30.
  nodal value (lumped L2-projection, Appendix A):
      |sum_e int N_p q / sum_e int N_p|  if |phi_p| <= 0.9, else 0.
  gamma = (1/eta) sqrt( (1/n_DI) sum over the n_DI nodes with |phi_p| <= 0.9 of
          the squared nodal value );  gamma = 0 when n_DI = 0.
  v and phi at n+alpha.
beta (Section 2.2.1):  beta = int F'(phi) / int sqrt(F(phi)) with the same
  quadrature; beta = 0 when the denominator is 0.
"""
from __future__ import annotations

import numpy as np

from .fields import Problem, State


def l2_project(pb: Problem, fq: np.ndarray) -> np.ndarray:
    """Lumped L2-projection of quadrature values to nodes: int N_p f / int N_p."""
    m = pb.mesh
    num = m.integrate(fq, None)
    den = m.integrate(np.ones_like(fq), None)
    return num / den


def l2_project_gradient(pb: Problem, u: np.ndarray) -> np.ndarray:
    """(3, nn) nodal gradient of u by the same projection (Appendix A, Eq. bp)."""
    g = pb.mesh.grad(u)
    return np.stack([l2_project(pb, g[..., d]) for d in range(3)])


def mobility_nodal(pb: Problem, st: State, i: int):
    """(nodal |q| values (zero outside the interface band), band mask)."""
    m = pb.mesh
    xa = pb.at_alpha(st)
    _, gvq = pb.velocity(xa)
    gphi = m.grad(xa[pb.phi_comp(i)])
    n2 = gphi[..., 0] ** 2 + gphi[..., 1] ** 2 + gphi[..., 2] ** 2
    num = 0.0
    for j in range(3):
        for k in range(3):
            num = num + gphi[..., j] * gvq[j][..., k] * gphi[..., k]
    q = np.where(n2 < 1e-30, 0.0, num / np.where(n2 < 1e-30, 1.0, n2))
    val = np.abs(l2_project(pb, q))
    band = np.abs(xa[pb.phi_comp(i)]) <= 0.9
    return np.where(band, val, 0.0), band


def mobility(pb: Problem, st: State, i: int) -> float:
    val, band = mobility_nodal(pb, st, i)
    n_di = int(band.sum())
    if n_di == 0:
        return 0.0
    return float(np.sqrt((val[band] ** 2).sum() / n_di) / pb.desc.eta)


def beta(pb: Problem, st: State, i: int) -> float:
    m = pb.mesh
    phi = m.val(pb.at_alpha(st)[pb.phi_comp(i)])
    num = m.integrate_scalar(phi ** 3 - phi)
    den = m.integrate_scalar(0.5 * np.abs(phi ** 2 - 1.0))
    return 0.0 if den == 0.0 else num / den
