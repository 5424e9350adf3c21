"""Pins of the oracle's partitioned time step (Section 2.5)."""
import numpy as np
import pytest

from oracle import step
from oracle.fields import Problem, State
from tests.helpers import desc_small
from workloads import node_coords


def _two_phase_rest(n=4):
    d = desc_small(n=(n, n, n), dirichlet=False, n_fluid=1, n_solid=1)
    pb = Problem(d)
    X = node_coords(d)
    x = np.zeros((d.ncomp, d.nn))
    r = np.sqrt(((X - 0.45) ** 2).sum(0))
    x[5] = np.tanh((0.3 - r) / (np.sqrt(2) * 0.5 * d.eps))  # too sharp: relaxes
    x[4] = -x[5]
    x[pb.b_comp(0, 0): pb.b_comp(0, 3)] = 1.0
    return d, pb, State(x.copy(), x.copy(), np.zeros_like(x))


def test_step_at_rest_conserves_phase_mass_and_partition():
    """v = 0 (no forcing), fixed mobility: the velocity stays 0, the indicators relax
    with int phi^i conserved (beta, Section 2.2.1) and phi_2 = -phi_1 preserved."""
    d, pb, st = _two_phase_rest()
    m = pb.mesh
    mass0 = [m.integrate_scalar(m.val(st.x[4 + i])) for i in range(2)]
    opt = step.StepOptions(k_max=6, fixed_nl_iters=True, rtol=1e-12, fixed_gamma=[0.5, 0.5])
    x0 = st.x.copy()
    step.time_step(pb, st, opt)
    assert np.abs(st.xn[0:3]).max() < 1e-12
    for i in range(2):
        mass = m.integrate_scalar(m.val(st.xn[4 + i]))
        assert abs(mass - mass0[i]) < 1e-7 * np.abs(x0[4 + i]).sum() * np.prod(m.h)
    assert np.abs(st.xn[4] + st.xn[5]).max() < 1e-9
    assert np.abs(st.xn[5] - x0[5]).max() > 1e-3  # it did move
    # B stays the identity where nothing moves
    assert np.abs(st.xn[pb.b_comp(0, 0)] - 1.0).max() < 1e-10
    assert np.abs(st.xn[pb.b_comp(0, 3)]).max() < 1e-10


def test_cavity_step_converges():
    """Lid-driven cavity, 4^3: one step reaches the nonlinear tolerance of Section 2.5
    and the corrector gives dx/dt^{n+1} = (x^{n+1} - x^n)/dt (rho_inf = 0)."""
    d = desc_small(n=(4, 4, 4), n_fluid=1, n_solid=1)
    pb = Problem(d)
    X = node_coords(d)
    x = np.zeros((d.ncomp, d.nn))
    r = np.sqrt(((X - [0.6, 0.5, 0.5][0]) ** 2).sum(0))
    x[5] = np.tanh((0.25 - r) / (np.sqrt(2) * d.eps))
    x[4] = -x[5]
    x[pb.b_comp(0, 0): pb.b_comp(0, 3)] = 1.0
    st = State(x.copy(), x.copy(), np.zeros_like(x))
    info = step.time_step(pb, st, step.StepOptions(k_max=10))
    assert info.nl_iters < 10
    assert max(info.ratios[-1]) < 5e-4
    xprev = x
    assert np.allclose(st.xdn, (st.xn - xprev) / d.dt, rtol=1e-12, atol=1e-12)
    i, j, k = pb.mesh.ijk()
    assert np.all(st.xn[0, k == d.nz] == 1.0)
