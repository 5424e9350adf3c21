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


def _mirror_x(pb, x):
    """The state seen in the mirror x -> Lx - x: nodal fields re-indexed, v_x and the
    B components with one x index (B12, B13) change sign."""
    d = pb.desc
    y = x.reshape(x.shape[0], d.nz + 1, d.ny + 1, d.nx + 1)[:, :, :, ::-1].reshape(x.shape).copy()
    y[0] *= -1.0
    for s in range(pb.ns):
        y[pb.b_comp(s, 3)] *= -1.0  # B12
        y[pb.b_comp(s, 5)] *= -1.0  # B13
    return y


def _swap_xy(pb, x):
    """The state with the x and y axes exchanged: nodal fields transposed, v_x <-> v_y,
    B11 <-> B22 and B23 <-> B13 (order [11, 22, 33, 12, 23, 13])."""
    d = pb.desc
    y = x.reshape(x.shape[0], d.nz + 1, d.ny + 1, d.nx + 1).transpose(0, 1, 3, 2).reshape(x.shape).copy()
    y[[0, 1]] = y[[1, 0]]
    for s in range(pb.ns):
        a, b = pb.b_comp(s, 0), pb.b_comp(s, 1)
        y[[a, b]] = y[[b, a]]
        a, b = pb.b_comp(s, 4), pb.b_comp(s, 5)
        y[[a, b]] = y[[b, a]]
    return y


def test_falling_sphere_steps_keep_the_box_symmetries():
    """A heavier elastic sphere on the vertical axis of a closed no-slip box under
    gravity: the problem is unchanged by the mirrors x -> 1 - x, y -> 1 - y and by the
    exchange of x and y, so two time steps (Section 2.5) must return states with the
    same symmetries (up to the linear tolerance).  A dropped or mis-indexed term in one
    direction, a wrong sign of an off-diagonal B component or B components stored in
    the wrong order breaks one of them; the at-rest start makes every term of the
    momentum, Allen-Cahn and B equations take part by the second step."""
    from workloads import BC_DIRICHLET, FaceBC, MeshDesc, Phase
    phases = [Phase(rho=1.0, mu=0.02), Phase(rho=2.0, mu=0.02, mu_L=0.5, solid=True)]
    faces = [FaceBC(BC_DIRICHLET, (0.0, 0.0, 0.0), 0) for _ in range(6)]
    d = MeshDesc(4, 4, 4, 1.0, 1.0, 1.0, phases, (0.0, 0.0, -9.81), eps=0.375, eta=0.2, dt=0.02,
                 rho_inf=0.0, c_i=36.0, faces=faces, pin_node=0)
    pb = Problem(d)
    X = node_coords(d)
    x = np.zeros((d.ncomp, d.nn))
    r = np.sqrt((X[0] - 0.5) ** 2 + (X[1] - 0.5) ** 2 + (X[2] - 0.55) ** 2)
    x[5] = np.tanh((0.3 - r) / (np.sqrt(2) * d.eps))
    x[4] = -x[5]
    x[pb.b_comp(0, 0): pb.b_comp(0, 3)] = 1.0
    st = State(x.copy(), x.copy(), np.zeros_like(x))
    opt = step.StepOptions(k_max=3, fixed_nl_iters=True, rtol=1e-12, max_iter=4000)
    for _ in range(2):
        step.time_step(pb, st, opt)
    xs = st.xn
    assert np.abs(xs[2]).max() > 1e-4                         # the sphere moves
    assert np.abs(xs[pb.b_comp(0, 4)]).max() > 1e-8          # B23 is no longer zero
    scale = np.abs(xs).max(axis=1, keepdims=True) + 1e-300
    mirror_y = _swap_xy(pb, _mirror_x(pb, _swap_xy(pb, xs)))
    for name, img in (("mirror x", _mirror_x(pb, xs)), ("mirror y", mirror_y), ("swap x y", _swap_xy(pb, xs))):
        err = (np.abs(img - xs) / scale).max()
        assert err < 1e-8, (name, err)
