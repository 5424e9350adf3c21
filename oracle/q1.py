"""Q1 hexahedral finite elements on a uniform box, 2x2x2 Gauss quadrature (oracle).

Test infrastructure only (see oracle/__init__.py).

The paper discretises with linear elements (Section 2.1.2); on the uniform
hexahedral meshes used here the trial/test space is trilinear (Q1).  Quadrature is
2-point Gauss-Legendre per axis (points +-1/sqrt(3), weights 1), exact for the
trilinear mass and stiffness integrands.

Conventions:
  node n = i + (nx+1)*(j + (ny+1)*k)
  element e = ex + nx*(ey + ny*ez)
  corner a = ax + 2*ay + 4*az, node of corner a = node(ex+ax, ey+ay, ez+az)
  quadrature point q = qx + 2*qy + 4*qz at xi = (g[qx], g[qy], g[qz]), g = (-1/sqrt3, +1/sqrt3)
"""
from __future__ import annotations

import numpy as np

GAUSS = np.array([-1.0 / np.sqrt(3.0), 1.0 / np.sqrt(3.0)])


def corner_signs() -> np.ndarray:
    """(8,3) reference-coordinate sign of each corner: -1 at xi=-1, +1 at xi=+1."""
    s = np.empty((8, 3))
    for a in range(8):
        s[a] = [2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
    return s


def gauss_points() -> np.ndarray:
    """(8,3) reference coordinates of the quadrature points."""
    p = np.empty((8, 3))
    for q in range(8):
        p[q] = [GAUSS[q & 1], GAUSS[(q >> 1) & 1], GAUSS[(q >> 2) & 1]]
    return p


def shape_values(xi: np.ndarray) -> np.ndarray:
    """Trilinear shape functions N_a(xi) = prod_d (1 + s_ad xi_d)/2 -> (npts, 8)."""
    s = corner_signs()
    return np.prod((1.0 + s[None, :, :] * xi[:, None, :]) / 2.0, axis=2)


def shape_gradients(xi: np.ndarray, h) -> np.ndarray:
    """Physical gradients dN_a/dx_d on an element of size h -> (npts, 8, 3).

    x_d = x0_d + (1 + xi_d) h_d / 2, so d xi_d / d x_d = 2 / h_d.
    """
    s = corner_signs()
    lin = (1.0 + s[None, :, :] * xi[:, None, :]) / 2.0  # (npts, 8, 3)
    out = np.empty((xi.shape[0], 8, 3))
    for d in range(3):
        others = [e for e in range(3) if e != d]
        out[:, :, d] = (s[None, :, d] / 2.0) * (2.0 / h[d]) * lin[:, :, others[0]] * lin[:, :, others[1]]
    return out


class Q1Mesh:
    """Uniform Q1 mesh with per-element gather and scatter."""

    def __init__(self, nx: int, ny: int, nz: int, lx: float, ly: float, lz: float):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.h = (lx / nx, ly / ny, lz / nz)
        self.nn = (nx + 1) * (ny + 1) * (nz + 1)
        self.ne = nx * ny * nz
        ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        # element order: ex fastest
        ex = ex.transpose(2, 1, 0).ravel()
        ey = ey.transpose(2, 1, 0).ravel()
        ez = ez.transpose(2, 1, 0).ravel()
        conn = np.empty((self.ne, 8), dtype=np.int64)
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            conn[:, a] = (ex + ax) + (nx + 1) * ((ey + ay) + (ny + 1) * (ez + az))
        self.conn = conn
        xi = gauss_points()
        self.N = shape_values(xi)            # (8q, 8a)
        self.dN = shape_gradients(xi, self.h)  # (8q, 8a, 3)
        # |det J| * Gauss weight (all weights are 1)
        self.wq = self.h[0] * self.h[1] * self.h[2] / 8.0

    # ---- interpolation to quadrature points
    def val(self, u: np.ndarray) -> np.ndarray:
        """Nodal (nn,) -> (ne, 8q) values at quadrature points."""
        return u[self.conn] @ self.N.T

    def grad(self, u: np.ndarray) -> np.ndarray:
        """Nodal (nn,) -> (ne, 8q, 3) gradients at quadrature points."""
        return np.einsum("ea,qad->eqd", u[self.conn], self.dN)

    # ---- weak-form assembly
    def integrate(self, f=None, g=None) -> np.ndarray:
        """Nodal r_a = sum_e sum_q w (N_a f + grad N_a . g).

        f: (ne, 8q) coefficient of the test function; g: (ne, 8q, 3) coefficient of
        its gradient.  Either may be None.
        """
        c = np.zeros((self.ne, 8))
        if f is not None:
            c += f @ self.N
        if g is not None:
            c += np.einsum("eqd,qad->ea", g, self.dN)
        c *= self.wq
        return np.bincount(self.conn.ravel(), weights=c.ravel(), minlength=self.nn)

    def integrate_scalar(self, f: np.ndarray) -> float:
        """sum_e sum_q w f(e,q) - the quadrature of a field over the domain."""
        return float(f.sum() * self.wq)

    def ijk(self):
        """(3, nn) integer node indices."""
        n = np.arange(self.nn)
        i = n % (self.nx + 1)
        j = (n // (self.nx + 1)) % (self.ny + 1)
        k = n // ((self.nx + 1) * (self.ny + 1))
        return np.stack([i, j, k])
