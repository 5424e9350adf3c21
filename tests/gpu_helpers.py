"""Helpers for the GPU parity tests: run libfsi through its C ABI on torch tensors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_10348_gb300 import fsi  # noqa: E402

DEV = "cuda:0"


def T(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device=DEV)


class Gpu:
    """A mesh handle plus device copies of a state."""

    def __init__(self, desc, x1, xn, xdn):
        self.d = desc
        self.mesh = fsi.fsi_create_mesh(desc)
        fsi.fsi_set_stream(self.mesh)
        self.x, self.xn, self.xdn = T(x1), T(xn), T(xdn)

    def st(self):
        return self.x, self.xn, self.xdn

    def residual(self, block, n):
        r = torch.zeros(n, dtype=torch.float64, device=DEV)
        fsi.fsi_residual(self.mesh, block, *self.st(), r)
        torch.cuda.synchronize()
        return r.cpu().numpy()

    def jvp(self, block, dx, flags=fsi.FSI_ELASTIC_AUG):
        y = torch.zeros(dx.size, dtype=torch.float64, device=DEV)
        fsi.fsi_jvp(self.mesh, block, *self.st(), T(dx.ravel()), y, flags)
        torch.cuda.synchronize()
        return y.cpu().numpy()

    def diag(self, block, n, flags=fsi.FSI_ELASTIC_AUG):
        y = torch.zeros(n, dtype=torch.float64, device=DEV)
        fsi.fsi_diag(self.mesh, block, *self.st(), y, flags)
        torch.cuda.synchronize()
        return y.cpu().numpy()


def relmax(a, b):
    """max |a - b| / max |b|."""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))
