"""Generalized-alpha time integration for first-order systems (oracle).

Test infrastructure only (see oracle/__init__.py).

Section 2.1.2 (generalized-alpha equations):
  phi^{n+1}        = phi^n + dt dphi^n + dt*vs*(dphi^{n+1} - dphi^n)
  dphi^{n+alpha_m} = dphi^n + alpha_m (dphi^{n+1} - dphi^n)
  phi^{n+alpha}    = phi^n + alpha (phi^{n+1} - phi^n)
  alpha = 1/(1+rho_inf), alpha_m = (3-rho_inf)/(2(1+rho_inf)), vs = 1/2 + alpha_m - alpha
The Newton unknown is phi^{n+1}; dphi^{n+1} follows from the first relation.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class GenAlpha:
    alpha: float
    alpha_m: float
    vs: float  # the paper's varsigma (written gamma in Appendix B)
    dt: float

    @staticmethod
    def from_rho_inf(rho_inf: float, dt: float) -> "GenAlpha":
        alpha = 1.0 / (1.0 + rho_inf)
        alpha_m = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf)
        vs = 0.5 + alpha_m - alpha
        return GenAlpha(alpha, alpha_m, vs, dt)

    def at_alpha(self, x1, xn):
        """x^{n+alpha}."""
        return xn + self.alpha * (x1 - xn)

    def xdot_np1(self, x1, xn, xdn):
        """dx^{n+1} solved from x^{n+1} = x^n + dt dx^n + dt vs (dx^{n+1} - dx^n)."""
        return xdn + (x1 - xn - self.dt * xdn) / (self.vs * self.dt)

    def xdot_at_alpha_m(self, x1, xn, xdn):
        """dx^{n+alpha_m} = dx^n + alpha_m (dx^{n+1} - dx^n)."""
        return xdn + self.alpha_m * (self.xdot_np1(x1, xn, xdn) - xdn)

    @property
    def c_mass(self) -> float:
        """d(dx^{n+alpha_m}) / d(x^{n+1}) = alpha_m / (vs dt)."""
        return self.alpha_m / (self.vs * self.dt)

    @property
    def c_elastic(self) -> float:
        """alpha vs dt / alpha_m: dB^{n+alpha} per unit dB/dt^{n+alpha_m} (Section 2.4)."""
        return self.alpha * self.vs * self.dt / self.alpha_m
