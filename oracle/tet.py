"""Linear (P1) tetrahedra: the element of the paper's falling-sphere and ship-ice meshes
(Sections 5.3 and 6) (oracle).

Test infrastructure only (see oracle/__init__.py).

The mesh keeps the node set, node numbering and boundary description of a box grid
(so the Dirichlet sets of oracle/bc.py apply unchanged) and splits every grid cell
into six tetrahedra around its diagonal from corner 0 to corner 7 (corner a = ax + 2ay
+ 4az), one per ordering of the three axes; every cell uses the same split, so the
tetrahedra of neighbouring cells share whole faces.  Interior nodes may be moved by a
seeded fraction of the spacing (`jitter`) to make every element different.

On a tetrahedron with vertices x_0..x_3 the shape functions are the barycentric
coordinates lambda_a, with constant gradients; quadrature is the symmetric 4-point
rule (barycentric points (a, b, b, b) and permutations, a = (5 + 3 sqrt5)/20,
b = (5 - sqrt5)/20, weights |T|/4), exact for quadratic integrands.  The stabilisation
metric is G = sum_k grad(xi_k) grad(xi_k)^T over the reference coordinates
xi_k = lambda_k, k = 1..3 (the reference element is the unit right tetrahedron), so
v.Gv, G:G and tr G are per element.

The interface matches oracle/q1.py's Q1Mesh (val, grad, integrate, integrate_scalar,
ijk), so the weak forms of ns.py, ac.py, cgt.py and mobility.py evaluate unchanged on
it through TetProblem.
"""
from __future__ import annotations


import numpy as np

from workloads import MeshDesc, tet_box_mesh  # the seeded input mesh

from .fields import Problem

_A = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
_B = (5.0 - np.sqrt(5.0)) / 20.0
QBARY = np.array([[_A, _B, _B, _B], [_B, _A, _B, _B], [_B, _B, _A, _B], [_B, _B, _B, _A]])  # (4q, 4a)


class TetMesh:
    """P1 tetrahedral mesh of a box grid's nodes."""

    def __init__(self, desc: MeshDesc, jitter: float = 0.0, seed: int = 0):
        nx, ny, nz = desc.nx, desc.ny, desc.nz
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nn = (nx + 1) * (ny + 1) * (nz + 1)
        h = desc.h
        self.h = h
        X, conn = tet_box_mesh(desc, jitter, seed)  # element e = 6 * cell + t, positive orientation
        self.X = X
        self.conn = conn
        self.ne = conn.shape[0]
        J = np.stack([X[:, conn[:, a]].T - X[:, conn[:, 0]].T for a in (1, 2, 3)], axis=2)
        self.vol = np.linalg.det(J) / 6.0
        # barycentric gradients: rows of J^{-1} are grad(lambda_1..3); grad(lambda_0) = -sum
        Jinv = np.linalg.inv(J)                      # (ne, 3, 3): d xi_k / d x_j = Jinv[k, j]
        g = np.empty((self.ne, 4, 3))
        g[:, 1:, :] = Jinv
        g[:, 0, :] = -Jinv.sum(axis=1)
        self.dNe = g                                 # (ne, 4a, 3)
        self.G = np.einsum("eki,ekj->eij", Jinv, Jinv)  # (ne, 3, 3)
        self.N = QBARY.copy()                        # (4q, 4a)
        self.wq = self.vol / 4.0                     # (ne,)

    def ijk(self):
        n = np.arange(self.nn)
        i = n % (self.nx + 1)
        j = (n // (self.nx + 1)) % (self.ny + 1)
        k = n // ((self.nx + 1) * (self.ny + 1))
        return np.stack([i, j, k])

    def val(self, u: np.ndarray) -> np.ndarray:
        """Nodal (nn,) -> (ne, 4q) values at the quadrature points."""
        return u[self.conn] @ self.N.T

    def grad(self, u: np.ndarray) -> np.ndarray:
        """Nodal (nn,) -> (ne, 4q, 3) gradients (constant on each element)."""
        g = np.einsum("ea,ead->ed", u[self.conn], self.dNe)
        return np.repeat(g[:, None, :], 4, axis=1)

    def integrate(self, f=None, g=None) -> np.ndarray:
        """Nodal r_a = sum_e sum_q w_e (N_a f + grad N_a . g)."""
        c = np.zeros((self.ne, 4))
        if f is not None:
            c += f @ self.N
        if g is not None:
            c += np.einsum("eqd,ead->ea", g, self.dNe)
        c *= self.wq[:, None]
        return np.bincount(self.conn.ravel(), weights=c.ravel(), minlength=self.nn)

    def integrate_scalar(self, f: np.ndarray) -> float:
        return float((f * self.wq[:, None]).sum())


class TetProblem(Problem):
    """Problem on P1 tetrahedra: the same weak forms with the per-element metric."""

    def __init__(self, desc: MeshDesc, jitter: float = 0.0, seed: int = 0):
        super().__init__(desc)
        self.mesh = TetMesh(desc, jitter, seed)
        G = self.mesh.G
        self.GG = (G ** 2).sum(axis=(1, 2))[:, None]           # (ne, 1)
        self.trG = np.trace(G, axis1=1, axis2=2)[:, None]      # (ne, 1)

    def vGv(self, vq):
        """v . G v at the quadrature points; vq (3, ne, 4q)."""
        return np.einsum("ieq,eij,jeq->eq", vq, self.mesh.G, vq)
