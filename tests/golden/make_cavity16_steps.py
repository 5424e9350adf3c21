"""Writes tests/golden/cavity16_steps.npz: the oracle's trajectory of the 16^3 lid-driven
cavity with the elastic sphere (Sections 5.1-5.2 geometry and materials on Q1 hexes),
five partitioned time steps of exactly five nonlinear iterations each (Section 2.5),
every block solve exact (sparse LU of the probed block Jacobian).

Calls only the oracle and the seeded workload description.  Stored: the initial state
x0 (phases from the grid-cell initialisation of Section 3), x^n after each step and
dx/dt^n after the last.  Run from the repository root:  python tests/golden/make_cavity16_steps.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import step  # noqa: E402
from oracle.fields import Problem, State  # noqa: E402
from oracle.gridcell import apply_rules, signed_distance_phi  # noqa: E402
from workloads import cavity16  # noqa: E402

STEPS = 5
K = 5


def initial_state(wl):
    d = wl.desc
    phi, _ = signed_distance_phi(d, wl.surfaces[0], d.eps, wl.grid_cells)
    x = np.zeros((d.ncomp, d.nn))
    x[4:4 + d.n_phase] = apply_rules(d, {0: phi}, wl.rules, d.eps)
    x[4 + d.n_phase: 4 + d.n_phase + 3] = 1.0
    return x


def main():
    wl = cavity16()
    d = wl.desc
    x0 = initial_state(wl)
    st = State(x0.copy(), x0.copy(), np.zeros_like(x0))
    pb = Problem(d)
    xs, xds = [], []
    for s in range(STEPS):
        t0 = time.time()
        info = step.time_step(pb, st, step.StepOptions(k_max=K, fixed_nl_iters=True, direct=True))
        xs.append(st.xn.copy())
        xds.append(st.xdn.copy())
        print(f"step {s + 1}: {time.time() - t0:.1f} s, ratios {info.ratios[-1]}", flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity16_steps.npz")
    np.savez_compressed(out, x0=x0, xn=np.array(xs), xdn_last=xds[-1], k=K)
    print("wrote", out)


if __name__ == "__main__":
    main()
