"""The pressure level of the enclosed cavity, and why its NS solves are taken without the
pin row.

With a Dirichlet velocity on every face, constant pressure is a null mode of the NS
Jacobian (Section 2.1.2's system; the pressure appears through its gradient and
through boundary rows that are all velocity rows) and the continuity rows sum to the
boundary flux of the velocity increment.  The pin row p = 0 at node 0 removes the null
mode but leaves a near-singular one: the residual component constant on the continuity
rows can only be removed through the lost continuity equation of the pin node.  Under
Jacobi GMRES(30) that component dominates the residual and converges far more slowly
than the rest.  Keeping the pin node's continuity equation (a consistent singular
system) and shifting the pressure afterwards gives the same Newton step."""
import copy

import numpy as np
import pytest

from oracle import blocks, step
from oracle.assemble import assemble
from oracle.fields import Problem, State
from oracle.gmres import gmres
from oracle.gridcell import apply_rules, signed_distance_phi
from workloads import cavity


def _initial(n):
    wl = cavity(n)
    d = wl.desc
    phi, _ = signed_distance_phi(d, wl.surfaces[0], d.eps, wl.grid_cells)
    x = np.zeros((d.ncomp, d.nn))
    x[4:4 + d.n_phase] = apply_rules(d, {0: phi}, wl.rules, d.eps)
    x[4 + d.n_phase: 4 + d.n_phase + 3] = 1.0
    return d, State(x.copy(), x.copy(), np.zeros_like(x))


def _unpinned(d):
    d2 = copy.copy(d)
    d2.pin_node = -1
    return d2


def test_pin_shift_step_equals_pinned_step():
    """Two nonlinear iterations of a 6^3 cavity step: exact pinned solves against GMRES on
    the unpinned system plus the shift, every field to 1e-10."""
    d, sa = _initial(6)
    _, sb = _initial(6)
    step.time_step(Problem(d), sa, step.StepOptions(k_max=2, fixed_nl_iters=True, direct=True))
    step.time_step(Problem(d), sb, step.StepOptions(k_max=2, fixed_nl_iters=True, rtol=1e-13, max_iter=5000,
                                                    pin_shift=True))
    assert sb.xn[3, d.pin_node] == 0.0
    for sl in (slice(0, 3), slice(3, 4), slice(4, 6), slice(6, 12)):
        assert np.linalg.norm(sa.xn[sl] - sb.xn[sl]) <= 1e-10 * np.linalg.norm(sa.xn[sl])


def test_unpinned_system_is_singular_and_consistent():
    """Constant pressure is in the null space of the unpinned Jacobian, and the Newton
    right-hand side of a state meeting the velocity conditions is orthogonal to the left
    null vector (ones on the continuity rows; the Dirichlet rows of the residual are 0)."""
    d, st = _initial(5)
    pb = Problem(d)
    step.predictor(pb, st)
    pu = Problem(_unpinned(d))
    A = assemble(pu, st, "ns")
    nn = d.nn
    ones_p = np.zeros(4 * nn)
    ones_p[3 * nn:] = 1.0
    assert np.linalg.norm(A @ ones_p) <= 1e-14 * abs(A).sum(axis=1).max() * np.sqrt(nn)
    b = -blocks.residual(pu, st, "ns")
    y = np.zeros(4 * nn)
    y[3 * nn:] = 1.0
    assert np.linalg.norm(b) > 0.0
    assert abs(y @ b) <= 1e-14 * np.abs(b).sum()


@pytest.fixture(scope="module")
def cavity16_ns():
    d, st = _initial(16)
    pb = Problem(d)
    step.predictor(pb, st)
    A = assemble(pb, st, "ns")
    b = -blocks.residual(pb, st, "ns")
    pu = Problem(_unpinned(d))
    Au = assemble(pu, st, "ns")
    bu = -blocks.residual(pu, st, "ns")
    return d, A, b, Au, bu


def test_pin_row_slows_jacobi_gmres_on_the_constant_continuity_mode(cavity16_ns):
    """First Newton system of the 16^3 cavity: Jacobi GMRES(30) reaches 1e-12 within 150
    iterations without the pin row; with it, 300 iterations leave more than 1e-8, and
    that residual lives on the continuity rows as a near-constant vector."""
    d, A, b, Au, bu = cavity16_ns
    _, it_u, rel_u = gmres(lambda u: Au @ u, bu, 1.0 / Au.diagonal(), 30, 1e-12, 150)
    assert rel_u <= 1e-12, (it_u, rel_u)
    x, it_p, rel_p = gmres(lambda u: A @ u, b, 1.0 / A.diagonal(), 30, 1e-12, 300)
    assert rel_p > 1e-8
    r = (b - A @ x).reshape(4, d.nn)
    rc = r[3]
    assert np.linalg.norm(rc) > 0.9 * np.linalg.norm(r)
    assert abs(rc.sum()) > 0.9 * np.sqrt(d.nn) * np.linalg.norm(rc)
