"""Linear tetrahedra on the GPU (csrc/tet.cu) against the oracle (oracle/tet.py).

Meshes: six tetrahedra per box cell around the cell diagonal, interior nodes jittered
by up to a quarter of the spacing, so every element has its own shape and metric.  The
NS, Allen-Cahn and B residuals, products (NS with and without the solid-stress
linearization) and Jacobi diagonals agree with the oracle to 1e-10 of the largest entry
(the two sum the element contributions in different orders), gamma and beta to 1e-11; a
float64 GMRES solve of the NS block meets the oracle's exact solve, and whole partitioned
steps match the oracle's steps with exact block solves."""
import numpy as np
import pytest

from tests.gpu_helpers import DEV, T, relmax

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from oracle import blocks, diag, ns  # noqa: E402
from oracle.assemble import assemble, direct_solve  # noqa: E402
from oracle.fields import State  # noqa: E402
from oracle.tet import TetProblem  # noqa: E402
from paper_2402_10348_gb300 import fsi  # noqa: E402
from tests.helpers import desc_small  # noqa: E402
from workloads import random_state  # noqa: E402

TOL = 1e-10
CASES = {
    "ragged_one_solid": dict(n=(9, 7, 6), L=(1.0, 0.8, 0.7), n_fluid=1, n_solid=1),
    "two_solids_gravity": dict(n=(5, 6, 4), n_fluid=2, n_solid=2, gravity=(0.0, 0.0, -9.81), rho_inf=0.5),
}


def _setup(case, seed=0):
    d = desc_small(**CASES[case])
    pb = TetProblem(d, jitter=0.25, seed=seed + 1)
    x1, xn, xdn = random_state(d, seed)
    mesh = fsi.fsi_create_tet_mesh(d, pb.mesh.X, pb.mesh.conn)
    fsi.fsi_set_stream(mesh)
    return d, pb, State(x1, xn, xdn), mesh, (T(x1), T(xn), T(xdn))


@pytest.mark.parametrize("case", list(CASES))
def test_tet_ns_residual_product_and_diagonal(case):
    d, pb, st, mesh, dst = _setup(case)
    n = 4 * d.nn
    r = torch.zeros(n, dtype=torch.float64, device=DEV)
    fsi.fsi_residual(mesh, fsi.FSI_BLOCK_NS, *dst, r)
    assert relmax(r.cpu().numpy(), ns.ns_residual(pb, st).ravel()) <= TOL
    dx = np.random.default_rng(3).normal(size=(4, d.nn))
    for aug in (True, False):
        y = torch.zeros(n, dtype=torch.float64, device=DEV)
        fsi.fsi_jvp(mesh, fsi.FSI_BLOCK_NS, *dst, T(dx.ravel()), y, fsi.FSI_ELASTIC_AUG if aug else 0)
        assert relmax(y.cpu().numpy(), ns.ns_jvp(pb, st, dx, elastic_aug=aug).ravel()) <= TOL, aug
    dg = torch.zeros(n, dtype=torch.float64, device=DEV)
    fsi.fsi_diag(mesh, fsi.FSI_BLOCK_NS, *dst, dg, fsi.FSI_ELASTIC_AUG)
    torch.cuda.synchronize()
    assert relmax(dg.cpu().numpy(), diag.block_diagonal(pb, st, "ns")) <= TOL


def test_tet_ns_gmres_meets_the_exact_solve():
    d, pb, st, mesh, dst = _setup("ragged_one_solid", seed=4)
    rhs = -blocks.residual(pb, st, "ns")
    exact = direct_solve(assemble(pb, st, "ns"), rhs)
    sol = torch.zeros(rhs.size, dtype=torch.float64, device=DEV)
    o = fsi.solve_opts(m=30, rtol=1e-12, max_iter=6000)
    o.flags |= fsi.FSI_NO_STALL_STOP
    info = fsi.fsi_gmres(mesh, fsi.FSI_BLOCK_NS, *dst, T(rhs), sol, o)
    torch.cuda.synchronize()
    got = sol.cpu().numpy()
    assert info.rel_res <= 1e-12
    assert np.linalg.norm(rhs - blocks.jvp(pb, st, "ns", got)) <= 1e-11 * np.linalg.norm(rhs)
    assert np.linalg.norm(got - exact) <= 1e-6 * np.linalg.norm(exact)


def test_tet_mesh_rejects_bad_elements_and_structured_calls():
    d = desc_small(n=(2, 2, 2))
    pb = TetProblem(d)
    X, conn = pb.mesh.X, pb.mesh.conn.copy()
    flipped = conn.copy()
    flipped[3] = flipped[3][[0, 2, 1, 3]]
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_create_tet_mesh(d, X, flipped)
    assert e.value.code == fsi.FSI_EINVAL and "non-positive volume" in str(e.value)
    bad = conn.copy()
    bad[0, 0] = d.nn
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_create_tet_mesh(d, X, bad)
    assert e.value.code == fsi.FSI_EINVAL and "out of range" in str(e.value)
    mesh = fsi.fsi_create_tet_mesh(d, X, conn)
    fsi.fsi_set_stream(mesh)
    x1, xn, xdn = (T(a) for a in random_state(d, 0))
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_batch_create([mesh], block=fsi.FSI_BLOCK_NS, m=30)
    assert e.value.code == fsi.FSI_EINVAL
    y = torch.zeros(4 * d.nn, dtype=torch.float64, device=DEV)
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_jvp(mesh, fsi.FSI_BLOCK_NS, x1, xn, xdn, y.clone(), y, fsi.FSI_ELASTIC_AUG | fsi.FSI_FP32)
    assert e.value.code == fsi.FSI_EINVAL


@pytest.mark.parametrize("block, name, ncomp", [(fsi.FSI_BLOCK_AC(1), ("ac", 1), 1), (fsi.FSI_BLOCK_B(0), ("b", 0), 6),
                                                (fsi.FSI_BLOCK_B(1), ("b", 1), 6)])
def test_tet_allen_cahn_and_b_blocks(block, name, ncomp):
    d, pb, st, mesh, dst = _setup("two_solids_gravity", seed=2)
    coeffs = {"gamma": {1: 0.45}, "beta": {1: -0.12}}
    fsi.fsi_set_ac_coeffs(mesh, 1, 0.45, -0.12)
    n = ncomp * d.nn
    r = torch.zeros(n, dtype=torch.float64, device=DEV)
    fsi.fsi_residual(mesh, block, *dst, r)
    dx = np.random.default_rng(5).normal(size=n)
    y = torch.zeros(n, dtype=torch.float64, device=DEV)
    fsi.fsi_jvp(mesh, block, *dst, T(dx), y)
    dg = torch.zeros(n, dtype=torch.float64, device=DEV)
    fsi.fsi_diag(mesh, block, *dst, dg)
    torch.cuda.synchronize()
    assert relmax(r.cpu().numpy(), blocks.residual(pb, st, name, coeffs)) <= TOL
    assert relmax(y.cpu().numpy(), blocks.jvp(pb, st, name, dx, coeffs)) <= TOL
    assert relmax(dg.cpu().numpy(), diag.block_diagonal(pb, st, name, coeffs)) <= TOL


def test_tet_gamma_beta():
    from oracle import mobility
    d, pb, st, mesh, dst = _setup("ragged_one_solid", seed=6)
    for i in range(d.n_phase):
        gb = fsi.fsi_update_ac_coeffs(mesh, i, *dst)
        assert gb[0] == pytest.approx(mobility.mobility(pb, st, i), rel=1e-11, abs=1e-300)
        assert gb[1] == pytest.approx(mobility.beta(pb, st, i), rel=1e-11, abs=1e-14)


def test_tet_time_steps_against_the_oracle():
    """Two partitioned steps (three fixed nonlinear iterations each) of a lid-driven cavity
    with an elastic sphere on jittered tetrahedra: the GPU (every block to rel-res 1e-12,
    the NS block with the pressure shift) against the oracle's exact block solves, every
    field to 1e-10."""
    from oracle import step as ostep
    from oracle.gridcell import apply_rules, signed_distance_phi
    from workloads import cavity
    wl = cavity(6)
    d = wl.desc
    pb = TetProblem(d, jitter=0.2, seed=7)
    phi, _ = signed_distance_phi(d, wl.surfaces[0], d.eps, wl.grid_cells)
    x = np.zeros((d.ncomp, d.nn))
    x[4:4 + d.n_phase] = apply_rules(d, {0: phi}, wl.rules, d.eps)
    x[4 + d.n_phase: 4 + d.n_phase + 3] = 1.0
    ref = State(x.copy(), x.copy(), np.zeros_like(x))
    mesh = fsi.fsi_create_tet_mesh(d, pb.mesh.X, pb.mesh.conn)
    fsi.fsi_set_stream(mesh)
    g = [T(x), T(x), T(np.zeros_like(x))]
    o = fsi.solve_opts(m=30, rtol=1e-12, max_iter=6000)
    for s in range(2):
        info = fsi.fsi_step(mesh, *g, k_max=3, fixed_iters=True, solve=o)
        ostep.time_step(pb, ref, ostep.StepOptions(k_max=3, fixed_nl_iters=True, direct=True))
        got = g[1].cpu().numpy().reshape(d.ncomp, d.nn)
        assert info.nl_iters == 3
        for sl in (slice(0, 3), slice(3, 4), slice(4, 6), slice(6, 12)):
            e = np.linalg.norm(got[sl] - ref.xn[sl]) / np.linalg.norm(ref.xn[sl])
            assert e <= 1e-10, (s, sl, e)
