"""Sparse block Jacobians by probing, and the exact (direct) linear solve (oracle).

Test infrastructure only (see oracle/__init__.py).

A column of a block Jacobian is, by definition, J e_j.  On the Q1 mesh the row of
(node a, component c) couples only to nodes sharing an element with a (index
difference at most 1 per axis), so nodes whose (i mod 3, j mod 3, k mod 3) agree
never share a row: one product with the sum of the unit vectors of such a colour
and one component gives 27 disjoint sets of columns at once.  Each nonzero of the
product at row node r belongs to the unique probed node within +-1 of r per axis.
The assembled matrix equals the matrix-free product up to summation order.

`direct_solve` is the exact Newton step the iterative solvers approximate
(Section 2.5 solves J d = -R for every block): a sparse LU solve of the assembled
matrix (a library routine).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import blocks
from .fields import Problem, State


def assemble(pb: Problem, st: State, block, coeffs=None, elastic_aug: bool = True) -> sp.csr_matrix:
    comps = blocks.components(pb, block)
    nc = len(comps)
    m = pb.mesh
    nn = m.nn
    i, j, k = m.ijk()
    colour = (i % 3) + 3 * (j % 3) + 9 * (k % 3)
    nx1, ny1 = m.nx + 1, m.ny + 1
    rows, cols, vals = [], [], []
    for c in range(nc):
        for col in range(27):
            sel = colour == col
            if not sel.any():
                continue
            e = np.zeros((nc, nn))
            e[c, sel] = 1.0
            y = blocks.jvp(pb, st, block, e.ravel(), coeffs, elastic_aug).reshape(nc, nn)
            rr, rn = np.nonzero(y)
            ci, cj, ck = col % 3, (col // 3) % 3, col // 9
            # the probed node within +-1 of the row node along each axis
            si = i[rn] + ((ci - i[rn]) % 3 + 1) % 3 - 1
            sj = j[rn] + ((cj - j[rn]) % 3 + 1) % 3 - 1
            sk = k[rn] + ((ck - k[rn]) % 3 + 1) % 3 - 1
            rows.append(rr * nn + rn)
            cols.append(c * nn + si + nx1 * (sj + ny1 * sk))
            vals.append(y[rr, rn])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc * nn, nc * nn))


def direct_solve(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """x with A x = b by sparse LU (SuperLU)."""
    return spla.spsolve(A.tocsc(), b)
