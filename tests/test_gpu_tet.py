"""Linear tetrahedra on the GPU (csrc/tet.cu) against the oracle (oracle/tet.py).

Meshes: six tetrahedra per box cell around the cell diagonal, interior nodes jittered
by up to a quarter of the spacing, so every element has its own shape and metric.  The
NS residual, product (with and without the solid-stress linearization) and Jacobi
diagonal agree with the oracle to 1e-10 of the largest entry (the two sum the element
contributions in different orders); a float64 GMRES solve of the NS block meets the
oracle's exact solve of the same system."""
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


def test_tet_mesh_rejects_bad_elements_and_other_blocks():
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
    r = torch.zeros(d.nn, dtype=torch.float64, device=DEV)
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_residual(mesh, fsi.FSI_BLOCK_AC(0), x1, xn, xdn, r)
    assert e.value.code == fsi.FSI_EINVAL
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_step(mesh, x1, xn, xdn)
    assert e.value.code == fsi.FSI_EINVAL
