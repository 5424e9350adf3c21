"""State layout and quadrature-point fields shared by the oracle's operators.

Test infrastructure only (see oracle/__init__.py).

Nodal state: x (ncomp, nn) float64 with component planes
    0..2          velocity v
    3             pressure p
    4..4+N-1      phase indicators phi^i
    4+N+6s+c      component c of B^s, c in [B11, B22, B33, B12, B23, B13]
                  (the ordering of Section 2.5, second remark)
and the generalized-alpha history x^n and xdot^n of the same shape.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from workloads import MeshDesc

from .galpha import GenAlpha
from .q1 import Q1Mesh

# (row, col) of each stored B component
SYM = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]
# stored component index of B_kl
SYM_INDEX = np.array([[0, 3, 5], [3, 1, 4], [5, 4, 2]])


@dataclass
class State:
    x: np.ndarray    # x^{n+1}
    xn: np.ndarray   # x^n
    xdn: np.ndarray  # xdot^n


class Problem:
    def __init__(self, desc: MeshDesc):
        self.desc = desc
        self.mesh = Q1Mesh(desc.nx, desc.ny, desc.nz, desc.lx, desc.ly, desc.lz)
        self.ga = GenAlpha.from_rho_inf(desc.rho_inf, desc.dt)
        self.N = desc.n_phase
        self.solids = desc.solid_phases
        self.ns = len(self.solids)
        h = self.mesh.h
        # contravariant metric of the uniform hex map: G = diag(4/h^2)
        self.Gd = np.array([4.0 / (h[0] ** 2), 4.0 / (h[1] ** 2), 4.0 / (h[2] ** 2)])
        self.GG = float((self.Gd ** 2).sum())
        self.trG = float(self.Gd.sum())

    def phi_comp(self, i: int) -> int:
        return 4 + i

    def b_comp(self, s: int, c: int) -> int:
        return 4 + self.N + 6 * s + c

    def vGv(self, vq):
        """v . G v at quadrature points; vq (3, ne, 8)."""
        return self.Gd[0] * vq[0] ** 2 + self.Gd[1] * vq[1] ** 2 + self.Gd[2] * vq[2] ** 2

    # --------------------------------------------------------- interpolations
    def at_alpha(self, st: State) -> np.ndarray:
        return self.ga.at_alpha(st.x, st.xn)

    def at_alpha_m(self, st: State) -> np.ndarray:
        return self.ga.xdot_at_alpha_m(st.x, st.xn, st.xdn)

    def velocity(self, xa):
        m = self.mesh
        vq = np.stack([m.val(xa[k]) for k in range(3)])            # (3, ne, 8)
        gvq = np.stack([m.grad(xa[k]) for k in range(3)])          # (3, ne, 8, 3): d v_k / d x_j
        return vq, gvq

    def materials(self, xa):
        """Blended density and dynamic viscosity at quadrature points and the phase
        fractions alpha^i = (1 + phi^i)/2 (Section 2.1.1; viscosity read as the
        dynamic viscosity mu)."""
        m = self.mesh
        alphas = []
        rho = 0.0
        mu = 0.0
        for i, ph in enumerate(self.desc.phases):
            a = (1.0 + m.val(xa[self.phi_comp(i)])) / 2.0
            alphas.append(a)
            rho = rho + a * ph.rho
            mu = mu + a * ph.mu
        return rho, mu, alphas

    def b_tensor(self, xa, s: int, with_grad: bool):
        """Full symmetric B^s (3,3,ne,8) and optionally its gradient (3,3,ne,8,3)."""
        m = self.mesh
        comp = [m.val(xa[self.b_comp(s, c)]) for c in range(6)]
        B = np.empty((3, 3) + comp[0].shape)
        for k in range(3):
            for l in range(3):
                B[k, l] = comp[SYM_INDEX[k, l]]
        if not with_grad:
            return B, None
        gcomp = [m.grad(xa[self.b_comp(s, c)]) for c in range(6)]
        gB = np.empty((3, 3) + gcomp[0].shape)
        for k in range(3):
            for l in range(3):
                gB[k, l] = gcomp[SYM_INDEX[k, l]]
        return B, gB
