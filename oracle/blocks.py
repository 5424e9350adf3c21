"""Block bookkeeping for the partitioned solve (oracle).

Test infrastructure only (see oracle/__init__.py).

Blocks (Section 2.5): "ns" (v, p), ("ac", i) for phase indicator i, ("b", s) for the
left Cauchy-Green tensor of solid s.  A block vector is the block's component planes
of the nodal state, flattened component-major.
"""
from __future__ import annotations

import numpy as np

from . import ac, cgt, ns
from .fields import Problem, State


def components(pb: Problem, block) -> list:
    if block == "ns":
        return [0, 1, 2, 3]
    kind, idx = block
    if kind == "ac":
        return [pb.phi_comp(idx)]
    return [pb.b_comp(idx, c) for c in range(6)]


def all_blocks(pb: Problem) -> list:
    return ["ns"] + [("ac", i) for i in range(pb.N)] + [("b", s) for s in range(pb.ns)]


def residual(pb: Problem, st: State, block, coeffs=None, coef_state: State | None = None) -> np.ndarray:
    """Block residual as a flat vector.  coeffs: {"gamma": [...], "beta": [...]}."""
    if block == "ns":
        return ns.ns_residual(pb, st, coef_state).ravel()
    kind, idx = block
    if kind == "ac":
        return ac.ac_residual(pb, st, idx, coeffs["gamma"][idx], coeffs["beta"][idx], coef_state).ravel()
    return cgt.cgt_residual(pb, st, idx, coef_state).ravel()


def jvp(pb: Problem, st: State, block, dx_flat: np.ndarray, coeffs=None, elastic_aug: bool = True) -> np.ndarray:
    nn = pb.mesh.nn
    if block == "ns":
        return ns.ns_jvp(pb, st, dx_flat.reshape(4, nn), elastic_aug).ravel()
    kind, idx = block
    if kind == "ac":
        return ac.ac_jvp(pb, st, idx, coeffs["gamma"][idx], coeffs["beta"][idx], dx_flat.reshape(nn)).ravel()
    return cgt.cgt_jvp(pb, st, idx, dx_flat.reshape(6, nn)).ravel()
