"""Left Cauchy-Green tensor transport: residual and Jacobian-vector product (oracle).

Test infrastructure only (see oracle/__init__.py).

Strong form (Section 2.3.1), per solid s with alpha = alpha^s = (1+phi^s)/2:
  alpha (dB/dt + (v.grad) B - grad v B - B grad v^T) + (1 - alpha)(B - I) = 0,
  (grad v)_km = d v_k / d x_m.
Variational form (Eq. semiCGT, Section 2.3.2), alpha read as a field inside the
integrals, each of the six stored components [B11,B22,B33,B12,B23,B13] tested with
its own scalar test function:
  int N_a Rb_c + int tau_B (v.grad N_a) Rb_c,
  Rb = alpha (dB + (v.grad) B - grad v B - B grad v^T) + (1 - alpha)(B - I),
  tau_B = ((2/dt)^2 + v.G v)^(-1/2)  (the printed parameter has no exponent; it is
          read as a time scale like tau_m and tau_phi).
B at n+alpha, dB at n+alpha_m, v and phi^s at n+alpha (frozen in this block).
The residual is linear in B; the Jacobian-vector product is its derivative in
B^{n+1}.  No Dirichlet rows.
"""
from __future__ import annotations

import numpy as np

from .fields import SYM, Problem, State


def _common(pb: Problem, coef: State, s: int):
    m = pb.mesh
    xa = pb.at_alpha(coef)
    vq, gvq = pb.velocity(xa)
    alpha = (1.0 + m.val(xa[pb.phi_comp(pb.solids[s])])) / 2.0
    tau = (4.0 / pb.desc.dt ** 2 + pb.vGv(vq)) ** -0.5
    return vq, gvq, alpha, tau


def _transport(vq, gvq, B, gB, dB, alpha, recovery_shift: bool):
    """Rb (6, ne, 8) for a full tensor B (3,3,...) with gradient gB and rate dB."""
    out = []
    for (k, l) in SYM:
        conv = sum(vq[mm] * gB[k, l][..., mm] for mm in range(3))
        stretch = sum(gvq[k][..., mm] * B[mm, l] for mm in range(3)) + \
            sum(B[k, mm] * gvq[l][..., mm] for mm in range(3))
        rec = B[k, l] - (1.0 if (recovery_shift and k == l) else 0.0)
        out.append(alpha * (dB[k, l] + conv - stretch) + (1.0 - alpha) * rec)
    return out


def _full(comps):
    from .fields import SYM_INDEX
    B = np.empty((3, 3) + comps[0].shape)
    for k in range(3):
        for l in range(3):
            B[k, l] = comps[SYM_INDEX[k, l]]
    return B


def cgt_residual(pb: Problem, st: State, s: int, coef: State | None = None) -> np.ndarray:
    """(6, nn)."""
    coef = st if coef is None else coef
    m = pb.mesh
    vq, gvq, alpha, tau = _common(pb, coef, s)
    xa = pb.at_alpha(st)
    xd = pb.at_alpha_m(st)
    cs = [pb.b_comp(s, c) for c in range(6)]
    B = _full([m.val(xa[c]) for c in cs])
    gB = _full([m.grad(xa[c]) for c in cs])
    dB = _full([m.val(xd[c]) for c in cs])
    R = _transport(vq, gvq, B, gB, dB, alpha, recovery_shift=True)
    out = np.empty((6, m.nn))
    for c in range(6):
        g = np.stack([tau * vq[j] * R[c] for j in range(3)], axis=-1)
        out[c] = m.integrate(R[c], g)
    return out


def cgt_jvp(pb: Problem, st: State, s: int, dB_np1: np.ndarray) -> np.ndarray:
    """(6, nn) = J_B dB with dB_np1 (6, nn) increments of B^{n+1}."""
    m = pb.mesh
    ga = pb.ga
    vq, gvq, alpha, tau = _common(pb, st, s)
    Bt = _full([ga.alpha * m.val(dB_np1[c]) for c in range(6)])
    gBt = _full([ga.alpha * m.grad(dB_np1[c]) for c in range(6)])
    dBt = _full([ga.c_mass * m.val(dB_np1[c]) for c in range(6)])
    R = _transport(vq, gvq, Bt, gBt, dBt, alpha, recovery_shift=False)
    out = np.empty((6, m.nn))
    for c in range(6):
        g = np.stack([tau * vq[j] * R[c] for j in range(3)], axis=-1)
        out[c] = m.integrate(R[c], g)
    return out
