"""Pins of the oracle's probed block Jacobians and its exact linear solve.

The assembled matrix is pinned to the definition of a Jacobian column (J e_j for
every unit vector, brute force on a tiny mesh) and to the matrix-free product on a
ragged mesh; the direct solve to the linear system it solves and to GMRES."""
import numpy as np
import pytest

from oracle import blocks, step
from oracle.assemble import assemble, direct_solve
from oracle.fields import Problem, State
from oracle.gmres import gmres
from oracle.gridcell import apply_rules, signed_distance_phi
from tests.helpers import desc_small, state_of
from workloads import cavity

BLOCKS = ["ns", ("ac", 0), ("ac", 1), ("b", 0)]
COEFFS = {"gamma": {0: 0.7, 1: 0.3}, "beta": {0: 0.2, 1: -0.1}}


@pytest.mark.parametrize("block", BLOCKS)
def test_assembly_equals_unit_vector_columns(block):
    """Every column J e_j by brute force (one product per unknown) on a 2x2x2 mesh."""
    d = desc_small(n=(2, 2, 2))
    pb, st = Problem(d), state_of(d, 4)
    A = assemble(pb, st, block, COEFFS).toarray()
    n = A.shape[0]
    cols = np.empty_like(A)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols[:, j] = blocks.jvp(pb, st, block, e, COEFFS)
    assert np.array_equal(A, cols)


@pytest.mark.parametrize("block", BLOCKS)
def test_assembly_matches_matrix_free_product_on_ragged_mesh(block):
    d = desc_small(n=(5, 4, 7), L=(1.0, 0.8, 1.3))
    pb, st = Problem(d), state_of(d, 9)
    A = assemble(pb, st, block, COEFFS)
    u = np.random.default_rng(2).normal(size=A.shape[0])
    y = blocks.jvp(pb, st, block, u, COEFFS)
    assert np.linalg.norm(A @ u - y) <= 1e-14 * np.linalg.norm(y)


def test_direct_solve_solves_and_agrees_with_gmres():
    d = desc_small(n=(4, 5, 3))
    pb, st = Problem(d), state_of(d, 5)
    A = assemble(pb, st, "ns")
    b = -blocks.residual(pb, st, "ns")
    x = direct_solve(A, b)
    assert np.linalg.norm(A @ x - b) <= 1e-13 * np.linalg.norm(b)
    xg, _, rel = gmres(lambda u: blocks.jvp(pb, st, "ns", u), b, 1.0 / A.diagonal(), 30, 1e-13, 5000)
    assert rel <= 1e-13
    assert np.linalg.norm(xg - x) <= 1e-9 * np.linalg.norm(x)


def test_time_step_with_direct_solves_matches_gmres_step():
    """One parity-mode cavity step: exact block solves and GMRES to 1e-13 give the same
    fields (the Newton iteration does not depend on which convergent solver runs)."""
    wl = cavity(5)
    d = wl.desc
    phi, _ = signed_distance_phi(d, wl.surfaces[0], d.eps, wl.grid_cells)
    x = np.zeros((d.ncomp, d.nn))
    x[4:4 + d.n_phase] = apply_rules(d, {0: phi}, wl.rules, d.eps)
    x[4 + d.n_phase: 4 + d.n_phase + 3] = 1.0
    sa = State(x.copy(), x.copy(), np.zeros_like(x))
    sb = State(x.copy(), x.copy(), np.zeros_like(x))
    step.time_step(Problem(d), sa, step.StepOptions(k_max=2, fixed_nl_iters=True, direct=True))
    step.time_step(Problem(d), sb, step.StepOptions(k_max=2, fixed_nl_iters=True, rtol=1e-13, max_iter=5000))
    for sl in (slice(0, 3), slice(3, 4), slice(4, 6), slice(6, 12)):
        assert np.linalg.norm(sa.xn[sl] - sb.xn[sl]) <= 1e-10 * np.linalg.norm(sb.xn[sl])
