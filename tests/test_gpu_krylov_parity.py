"""GMRES on the GPU against the oracle at sizes that reach the multi-CTA Krylov paths.

The B block of a 24 x 23 x 22 mesh has 82,800 unknowns: 324 basis chunks of 256, so
the fused update and second-pass kernels run on their full 304-CTA grids with a ragged
last chunk.  Each block system J x = -R is solved by the GPU (float64, and float32
inside float64 refinement; classical Gram-Schmidt with the DGKS second pass) and by the
oracle's modified Gram-Schmidt GMRES, both to rel-res 1e-12, and the solutions agree to
1e-9.  The GPU solution's residual is also recomputed with the oracle's own operator.
The state has no nodal noise, so every phase fraction lies in [0, 1] and the B block's
mass term (alpha c_mass + 1 - alpha) stays positive."""
import numpy as np
import pytest

from tests.gpu_helpers import DEV, Gpu, T

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from oracle import blocks, gmres  # noqa: E402
from oracle.fields import Problem, State  # noqa: E402
from paper_2402_10348_gb300 import fsi  # noqa: E402
from tests.helpers import desc_small  # noqa: E402
from workloads import random_state  # noqa: E402

COEFFS = {"gamma": {1: 0.4}, "beta": {1: 0.1}}
_REF = {}


@pytest.fixture(scope="module")
def system():
    d = desc_small(n=(24, 23, 22), n_fluid=1, n_solid=1)
    x1, xn, xdn = random_state(d, 11, noise=0.0)
    return d, Problem(d), State(x1, xn, xdn), Gpu(d, x1, xn, xdn)


def _oracle_solution(pb, st, block_name, coeffs):
    """Oracle GMRES(30) to 1e-12, right-scaled by the nodal mass coefficient of the block
    (any fixed positive diagonal: the solution does not depend on it)."""
    key = block_name
    if key not in _REF:
        rhs = -blocks.residual(pb, st, block_name, coeffs)
        a = (1.0 + st.x[pb.phi_comp(1)]) / 2.0
        if block_name[0] == "b":
            minv = np.tile(1.0 / (a * pb.ga.c_mass + (1.0 - a)), 6)
        else:
            minv = None
        ref, it, rel = gmres.gmres(lambda u: blocks.jvp(pb, st, block_name, u, coeffs), rhs, minv, m=30,
                                   rtol=1e-12, max_iter=600)
        assert rel <= 1e-12, (block_name, it, rel)
        _REF[key] = (rhs, ref)
    return _REF[key]


@pytest.mark.parametrize("block_name, block_id", [(("b", 0), fsi.FSI_BLOCK_B(0)), (("ac", 1), fsi.FSI_BLOCK_AC(1))])
@pytest.mark.parametrize("precision", [fsi.FSI_PREC_FP64, fsi.FSI_PREC_FP32_IR])
def test_block_gmres_against_oracle_on_full_grids(system, block_name, block_id, precision):
    d, pb, st, g = system
    coeffs = None
    if block_name[0] == "ac":
        fsi.fsi_set_ac_coeffs(g.mesh, 1, 0.4, 0.1)
        coeffs = COEFFS
    rhs, ref = _oracle_solution(pb, st, block_name, coeffs)
    sol = torch.zeros(rhs.size, dtype=torch.float64, device=DEV)
    o = fsi.solve_opts(m=30, rtol=1e-12, max_iter=6000, precision=precision, ir_inner_rtol=1e-3, ir_max=40)
    o.flags |= fsi.FSI_NO_STALL_STOP
    info = fsi.fsi_gmres(g.mesh, block_id, *g.st(), T(rhs), sol, o)
    torch.cuda.synchronize()
    got = sol.cpu().numpy()
    assert info.rel_res <= 1e-12
    true = np.linalg.norm(rhs - blocks.jvp(pb, st, block_name, got, coeffs)) / np.linalg.norm(rhs)
    assert true <= 1e-11, true
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
