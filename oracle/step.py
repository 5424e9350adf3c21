"""Partitioned block Newton time step (oracle).

Test infrastructure only (see oracle/__init__.py).

Section 2.1.2 (predictor-multicorrector) and Section 2.5:
  predictor:  x^{n+1} = x^n (velocity Dirichlet values imposed), generalized-alpha
              history unchanged;
  for k = 1..K_max (nonlinear iterations):
     NS block:     solve J_NS d = -R_NS, v,p += d          (Eq. LS_NS)
     each phase i: gamma^i, beta^i frozen at the current state,
                   solve J_phi d = -R_phi, phi^i += d       (Eq. LS_AC)
     each solid s: solve J_B d = -R_B, B^s += d             (Eq. LS_MC)
     stop when ||d_blk|| / ||x_blk|| < nl_tol for every block;
  corrector:  xdot^{n+1} from the generalized-alpha relation, then
              x^n <- x^{n+1}, xdot^n <- xdot^{n+1}.
Every block's linear system is solved by Jacobi-preconditioned GMRES(m) from 0, or
(option `direct`) exactly, by a sparse LU solve of the probed block Jacobian: the
Newton step that every convergent linear solver approaches.  Option `pin_shift`: on an
enclosed domain the NS step is computed from the system in which the pin node keeps
its continuity equation (singular, consistent) followed by the shift p -= p[pin]; in
exact arithmetic this is the pinned step.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field

import numpy as np

from . import blocks, mobility
from .bc import dirichlet
from .diag import block_diagonal
from .fields import Problem, State
from .assemble import assemble, direct_solve
from .gmres import gmres
from workloads import BC_DIRICHLET


@dataclass
class StepOptions:
    k_max: int = 5
    nl_tol: float = 5e-4
    m: int = 30
    rtol: float = 1e-8
    max_iter: int = 2000
    fixed_nl_iters: bool = False       # run exactly k_max iterations (parity mode)
    fixed_gamma: list | None = None    # per-phase gamma instead of the mobility model
    elastic_aug: bool = True
    direct: bool = False               # exact linear solves (sparse LU of the probed Jacobian)
    pin_shift: bool = False            # enclosed domain: NS solve keeps the pin node's continuity
                                       # equation, then p -= p[pin] (same Newton step)


@dataclass
class StepInfo:
    nl_iters: int = 0
    gmres_iters: dict = field(default_factory=dict)
    ratios: list = field(default_factory=list)
    gamma: list = field(default_factory=list)
    beta: list = field(default_factory=list)


def predictor(pb: Problem, st: State) -> None:
    st.x[:] = st.xn
    vmask, vD, pmask = dirichlet(pb.desc)
    for k in range(3):
        st.x[k, vmask] = vD[k, vmask]
    st.x[3, pmask] = 0.0


def corrector(pb: Problem, st: State) -> None:
    xd1 = pb.ga.xdot_np1(st.x, st.xn, st.xdn)
    st.xn[:] = st.x
    st.xdn[:] = xd1


def enclosed(desc) -> bool:
    """Every face has a Dirichlet velocity: constant pressure is a null mode of the NS
    Jacobian (the pressure appears only through its gradient and through boundary
    rows that are all velocity Dirichlet rows)."""
    return all(f.kind == BC_DIRICHLET for f in desc.faces)


def _unpinned(pb: Problem) -> Problem:
    d = copy.copy(pb.desc)
    d.pin_node = -1
    return Problem(d)


def solve_block(pb: Problem, st: State, block, opt: StepOptions, coeffs=None):
    if block == "ns" and opt.pin_shift and pb.desc.pin_node >= 0 and enclosed(pb.desc):
        if opt.direct:
            raise ValueError("pin_shift solves a singular system: it needs the iterative solver")
        # the pinned Newton step, reached through the singular but consistent system in
        # which the pin node keeps its continuity equation (x_p + dx_p is then fixed
        # only up to a constant, removed by the shift to p = 0 at the pin node)
        x_before = st.x[0:4].copy()
        _, it, rel = _solve(_unpinned(pb), st, block, opt, coeffs)
        st.x[3] -= st.x[3, pb.desc.pin_node]
        dx = float(np.linalg.norm(st.x[0:4] - x_before))
        xnorm = float(np.linalg.norm(st.x[0:4]))
        return dx / xnorm if xnorm > 0.0 else dx, it, rel
    return _solve(pb, st, block, opt, coeffs)


def _solve(pb: Problem, st: State, block, opt: StepOptions, coeffs=None):
    comps = blocks.components(pb, block)
    r = blocks.residual(pb, st, block, coeffs)
    if opt.direct:
        A = assemble(pb, st, block, coeffs, opt.elastic_aug)
        dx = direct_solve(A, -r)
        it = 0
        rel = float(np.linalg.norm(A @ dx + r)) / max(float(np.linalg.norm(r)), 1e-300)
    else:
        d = block_diagonal(pb, st, block, coeffs, opt.elastic_aug)
        minv = 1.0 / d
        dx, it, rel = gmres(lambda u: blocks.jvp(pb, st, block, u, coeffs, opt.elastic_aug),
                            -r, minv, opt.m, opt.rtol, opt.max_iter)
    nn = pb.mesh.nn
    dx = dx.reshape(len(comps), nn)
    st.x[comps] += dx
    xnorm = float(np.linalg.norm(st.x[comps]))
    ratio = float(np.linalg.norm(dx)) / xnorm if xnorm > 0.0 else float(np.linalg.norm(dx))
    return ratio, it, rel


def time_step(pb: Problem, st: State, opt: StepOptions) -> StepInfo:
    info = StepInfo()
    predictor(pb, st)
    for k in range(opt.k_max):
        ratios = []
        r, it, _ = solve_block(pb, st, "ns", opt)
        ratios.append(r)
        info.gmres_iters.setdefault("ns", []).append(it)
        gam, bet = [], []
        for i in range(pb.N):
            g = opt.fixed_gamma[i] if opt.fixed_gamma is not None else mobility.mobility(pb, st, i)
            b = mobility.beta(pb, st, i)
            gam.append(g)
            bet.append(b)
            coeffs = {"gamma": {i: g}, "beta": {i: b}}
            r, it, _ = solve_block(pb, st, ("ac", i), opt, coeffs)
            ratios.append(r)
            info.gmres_iters.setdefault(f"ac{i}", []).append(it)
        for s in range(pb.ns):
            r, it, _ = solve_block(pb, st, ("b", s), opt)
            ratios.append(r)
            info.gmres_iters.setdefault(f"b{s}", []).append(it)
        info.gamma.append(gam)
        info.beta.append(bet)
        info.ratios.append(ratios)
        info.nl_iters = k + 1
        if not opt.fixed_nl_iters and max(ratios) < opt.nl_tol:
            break
    corrector(pb, st)
    return info
