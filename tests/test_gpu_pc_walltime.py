"""The learned preconditioner against Jacobi in wall time on the 64^3 cavity's NS block.

Setup as a run uses it: one float64 time step harvests training pairs from its Jacobi
solves, synthetic multi-scale pairs (fsi_pc_add_smooth_pairs) are added at the state it
reaches, the linear U-Net is trained, and the next NS system at that state (unpinned, as
the step solves it) is solved to rel-res 1e-8 by Jacobi GMRES(30) and by flexible
GMRES(30) whose directions alternate between the network and Jacobi.  Both reach the
tolerance (checked with the float64 operator), the flexible solve without the Jacobi
fallback, in fewer iterations and less wall time (each solve timed after one untimed
run).  Measured on a GB300: about 160 against 480 iterations, 0.22 s against 0.47 s."""
import time

import numpy as np
import pytest

from tests.gpu_helpers import DEV

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from paper_2402_10348_gb300 import fsi  # noqa: E402
from workloads import cavity64, he_normal_weights  # noqa: E402


def _initial_state(mesh, wl):
    d = wl.desc
    nn = d.nn
    phi = torch.zeros(d.n_phase * nn, dtype=torch.float64, device=DEV)
    fsi.fsi_init_phases(mesh, wl.surfaces, wl.rules, wl.grid_cells, phi)
    x = torch.zeros(d.ncomp * nn, dtype=torch.float64, device=DEV)
    x[4 * nn:(4 + d.n_phase) * nn] = phi
    base = 4 + d.n_phase
    for s in range(d.n_solid):
        x[(base + 6 * s) * nn:(base + 6 * s + 3) * nn] = 1.0
    return x, x.clone(), torch.zeros_like(x)


def _timed(mesh, st, rhs, opts):
    sol = torch.zeros_like(rhs)
    fsi.fsi_gmres(mesh, fsi.FSI_BLOCK_NS, *st, rhs, sol, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = fsi.fsi_gmres(mesh, fsi.FSI_BLOCK_NS, *st, rhs, sol, opts)
    torch.cuda.synchronize()
    return info, time.perf_counter() - t0, sol


def test_learned_pc_beats_jacobi_in_wall_time_at_64():
    wl = cavity64()
    d = wl.desc
    mesh = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(mesh)
    st = _initial_state(mesh, wl)
    pc = fsi.fsi_pc_create(mesh, n_pairs_cap=512, linear=True, modulate=True)
    fsi.fsi_pc_set_weights(pc, he_normal_weights(pc.fan, 3))
    fsi.fsi_set_pc(mesh, pc)
    harvest = fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000)
    harvest.flags |= fsi.FSI_HARVEST
    fsi.fsi_step(mesh, *st, k_max=5, nl_tol=5e-4, solve=harvest)
    fsi.fsi_pc_add_smooth_pairs(pc, *st, 360, seed=1)
    npairs = fsi.fsi_pc_pairs(pc)
    assert npairs >= 360
    fsi.fsi_pc_fit_norm(pc)
    losses = fsi.fsi_pc_train(pc, np.random.default_rng(0).integers(0, npairs, size=4000), 2e-4)
    assert losses[-200:].mean() < 0.2

    fsi.fsi_set_pressure_pin(mesh, False)
    r = torch.zeros(4 * d.nn, dtype=torch.float64, device=DEV)
    fsi.fsi_residual(mesh, fsi.FSI_BLOCK_NS, *st, r)
    rhs = -r
    jac, tj, _ = _timed(mesh, st, rhs, fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000))
    o = fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000, precond=fsi.FSI_PC_LEARNED)
    o.flags |= fsi.FSI_PC_ALTERNATE
    lrn, tl, sol = _timed(mesh, st, rhs, o)
    t = torch.zeros_like(rhs)
    fsi.fsi_jvp(mesh, fsi.FSI_BLOCK_NS, *st, sol, t)
    torch.cuda.synchronize()
    true_rel = float(torch.linalg.norm(rhs - t) / torch.linalg.norm(rhs))
    print(f"Jacobi {jac.iterations} it {tj:.3f} s; learned {lrn.iterations} it {tl:.3f} s "
          f"(rel {lrn.rel_res:.2e}, true {true_rel:.2e}, fallback {lrn.fallback})")
    assert jac.rel_res <= 1e-8 and lrn.rel_res <= 1e-8 and true_rel <= 1.5e-8
    assert lrn.fallback == 0
    assert lrn.iterations < 0.7 * jac.iterations
    assert tl < 0.8 * tj
