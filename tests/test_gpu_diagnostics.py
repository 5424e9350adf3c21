"""Diagnostics on the GPU (csrc/diag.cu) against the oracle: the solid centre of mass of
Section 5.2 and the point tracking of Appendix C, on cubic and ragged meshes."""
import numpy as np
import pytest

from tests.gpu_helpers import DEV, T
from tests.helpers import desc_small

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from oracle import diagnostics  # noqa: E402
from oracle.fields import Problem  # noqa: E402
from paper_2402_10348_gb300 import fsi  # noqa: E402
from workloads import cavity, random_state  # noqa: E402


@pytest.mark.parametrize("d", [cavity(12).desc, desc_small(n=(7, 11, 5), L=(0.9, 1.3, 0.6)),
                               desc_small(n=(9, 4, 13), n_solid=2)])
def test_center_of_mass_matches_oracle(d):
    x1 = random_state(d, 3)[0]
    mesh = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(mesh)
    pb = Problem(d)
    for s in range(d.n_solid):
        got = np.array(fsi.fsi_center_of_mass(mesh, T(x1), s))
        ref = diagnostics.center_of_mass(pb, x1, s)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_track_points_matches_oracle():
    d = desc_small(n=(7, 11, 5), L=(0.9, 1.3, 0.6))
    x1 = random_state(d, 4)[0]
    mesh = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(mesh)
    rng = np.random.default_rng(5)
    L = np.array([d.lx, d.ly, d.lz])
    pts = rng.uniform(-0.1, 1.1, size=(5000, 3)) * L            # some outside the box
    X = diagnostics.node_xyz(Problem(d))
    pts = np.concatenate([pts, X[:, ::7].T, [[0.0, 0.0, 0.0], list(L)]])  # nodes and corners
    got = T(pts)
    fsi.fsi_track_points(mesh, T(x1), got)
    torch.cuda.synchronize()
    ref = diagnostics.track_points(Problem(d), x1, pts)
    assert np.abs(got.cpu().numpy() - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


def test_tracking_no_points_and_bad_solid():
    d = desc_small(n=(3, 3, 3))
    x1 = random_state(d, 1)[0]
    mesh = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(mesh)
    empty = torch.zeros((0, 3), dtype=torch.float64, device=DEV)
    fsi.fsi_track_points(mesh, T(x1), empty)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_center_of_mass(mesh, T(x1), 5)
