"""Diagnostics of a computed state (oracle): solid centre of mass and tracked points.

Test infrastructure only (see oracle/__init__.py).

Section 5.2 measures a solid by the centre of mass of its indicator,
    x_c = int x alpha^s dOmega / int alpha^s dOmega,   alpha^s = (1 + phi^s) / 2.
Appendix C follows a material point of a solid through an Eulerian solution: find
the element that holds it, interpolate the velocity there with that element's shape
functions, and move the point with it, every time step.

Readings (the paper works on linear tetrahedra; these meshes are uniform Q1 hexes):
  - both integrals use the 2x2x2 Gauss rule of the operators, which is exact here
    (alpha is trilinear and x linear in every element);
  - the element of a point follows from its coordinates, cell = floor(p / h), and the
    velocity is the trilinear Q1 interpolant of the nodal velocity of the new time
    level (v^{n+1}; with rho_inf = 0 that is v^{n+alpha});
  - one forward-Euler move per step:  p^{n+1} = p^n + dt v^{n+1}(p^n);
  - a point outside the box is first clamped onto it; a point on an interior element
    face belongs to the element above it, a point on an upper box face to the last
    element (the interpolant is continuous, so the choice does not change v).
"""
from __future__ import annotations

import numpy as np

from .fields import Problem


def node_xyz(pb: Problem) -> np.ndarray:
    """(3, nn) node coordinates."""
    m = pb.mesh
    ijk = m.ijk()
    return np.stack([ijk[d] * m.h[d] for d in range(3)]).astype(np.float64)


def center_of_mass(pb: Problem, x: np.ndarray, s: int) -> np.ndarray:
    """(3,) centre of mass of solid s (Section 5.2) from the state x (ncomp, nn)."""
    m = pb.mesh
    alpha = (1.0 + m.val(x[pb.phi_comp(pb.solids[s])])) / 2.0
    X = node_xyz(pb)
    mass = m.integrate_scalar(alpha)
    first = np.array([m.integrate_scalar(alpha * m.val(X[d])) for d in range(3)])
    return first / mass


def locate(pb: Problem, points: np.ndarray):
    """Element cell (n, 3) int and local coordinates (n, 3) in [0, 1] of each point
    (clamped onto the box first)."""
    m = pb.mesh
    d = pb.desc
    L = np.array([d.lx, d.ly, d.lz])
    nc = np.array([m.nx, m.ny, m.nz])
    h = np.array(m.h)
    p = np.clip(np.asarray(points, dtype=np.float64), 0.0, L)
    cell = np.minimum(np.floor(p / h).astype(np.int64), nc - 1)
    xi = (p - cell * h) / h
    return cell, xi


def interpolate_velocity(pb: Problem, x: np.ndarray, points: np.ndarray) -> np.ndarray:
    """(n, 3) trilinear interpolant of the nodal velocity x[0:3] at the points."""
    m = pb.mesh
    cell, xi = locate(pb, points)
    out = np.zeros((len(cell), 3))
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        w = ((xi[:, 0] if ax else 1.0 - xi[:, 0]) * (xi[:, 1] if ay else 1.0 - xi[:, 1]) *
             (xi[:, 2] if az else 1.0 - xi[:, 2]))
        node = (cell[:, 0] + ax) + (m.nx + 1) * ((cell[:, 1] + ay) + (m.ny + 1) * (cell[:, 2] + az))
        for k in range(3):
            out[:, k] += w * x[k, node]
    return out


def track_points(pb: Problem, x_np1: np.ndarray, points: np.ndarray) -> np.ndarray:
    """(n, 3) points moved by one step of Appendix C: p + dt v^{n+1}(p)."""
    p = np.asarray(points, dtype=np.float64)
    return p + pb.desc.dt * interpolate_velocity(pb, x_np1, p)
