"""Jacobi diagonal of a block Jacobian by probing (oracle).

Test infrastructure only (see oracle/__init__.py).

By definition d_i = e_i^T J e_i.  On the Q1 mesh row (node a, component c) of J only
couples to nodes that share an element with a, i.e. whose index differs by at most 1
in each direction.  Nodes whose (i mod 3, j mod 3, k mod 3) agree are therefore never
coupled, so J applied to the sum of the unit vectors of one such colour and one
component returns, at each of those nodes, exactly its own diagonal entry.
27 colours x (components) products give the whole diagonal.
"""
from __future__ import annotations

import numpy as np

from . import blocks
from .fields import Problem, State


def block_diagonal(pb: Problem, st: State, block, coeffs=None, elastic_aug: bool = True) -> np.ndarray:
    comps = blocks.components(pb, block)
    nc = len(comps)
    nn = pb.mesh.nn
    i, j, k = pb.mesh.ijk()
    colour = (i % 3) + 3 * (j % 3) + 9 * (k % 3)
    d = np.zeros((nc, nn))
    for c in range(nc):
        for col in range(27):
            sel = colour == col
            if not sel.any():
                continue
            e = np.zeros((nc, nn))
            e[c, sel] = 1.0
            y = blocks.jvp(pb, st, block, e.ravel(), coeffs, elastic_aug).reshape(nc, nn)
            d[c, sel] = y[c, sel]
    return d.ravel()
