"""The allocation-free gamma/beta entry point agrees with fsi_update_ac_coeffs.

fsi_gamma_beta_noalloc serves callers that cannot call cudaMalloc (code that must not
synchronise the device, or that runs under a framework allocator owning all device
memory): it keeps its per-CTA partial sums in a static device array instead of
allocating.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2402_10348_gb300 import fsi  # noqa: E402
from tests.helpers import desc_small  # noqa: E402
from workloads import random_state  # noqa: E402

DEV = "cuda:0"


def _state(d, seed):
    x1, xn, xdn = random_state(d, seed)
    return [torch.tensor(a.ravel(), dtype=torch.float64, device=DEV) for a in (x1, xn, xdn)]


@pytest.mark.parametrize("n", [(20, 17, 13), (6, 5, 4)])
def test_noalloc_matches_update_ac_coeffs_twice(n):
    d = desc_small(n=n, n_fluid=1, n_solid=1)  # rho_inf = 0: x^{n+alpha} = x^{n+1}
    x, xn, xdn = _state(d, 7)
    mesh = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(mesh)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=DEV)
    nn = d.nn
    for call in range(2):
        for i in range(d.n_phase):
            ref = fsi.fsi_update_ac_coeffs(mesh, i, x, xn, xdn)
            v = x[0:3 * nn]
            phi = x[(4 + i) * nn:(5 + i) * nn]
            rc = fsi.lib().fsi_gamma_beta_noalloc(
                ctypes.c_int32(d.nx), ctypes.c_int32(d.ny), ctypes.c_int32(d.nz), ctypes.c_double(d.lx),
                ctypes.c_double(d.ly), ctypes.c_double(d.lz), ctypes.c_double(d.eta),
                ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == fsi.FSI_OK, fsi.lib().fsi_last_error().decode()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert got[0] == pytest.approx(ref[0], rel=1e-12, abs=1e-300), (call, i)
            assert got[1] == pytest.approx(ref[1], rel=1e-12, abs=1e-14), (call, i)
            out.fill_(float("nan"))


def _raw_call(nx, ny, nz, v, phi, out):
    return fsi.lib().fsi_gamma_beta_noalloc(
        ctypes.c_int32(nx), ctypes.c_int32(ny), ctypes.c_int32(nz), ctypes.c_double(1.0), ctypes.c_double(1.0),
        ctypes.c_double(1.0), ctypes.c_double(0.2), ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_rejects_meshes_beyond_the_scratch():
    buf = torch.zeros(8, dtype=torch.float64, device=DEV)
    # 4096^3 and the int32 extreme would need far more than 16384 partial sums: the
    # library rejects them from the sizes alone, before any kernel runs (the binding
    # would already refuse the undersized tensors, so the C call is made directly)
    for n in (4096, 2 ** 31 - 1):
        rc = _raw_call(n, n, n, buf, buf, buf)
        assert rc == fsi.FSI_EINVAL
        assert "static scratch" in fsi.lib().fsi_last_error().decode()


def test_noalloc_binding_rejects_tensors_on_another_device(monkeypatch):
    """The kernel runs on the current device with that device's scratch, so tensors on
    any other GPU are refused by the binding (simulated: the current device is
    reported as another ordinal)."""
    d = desc_small(n=(4, 4, 4))
    x, _, _ = _state(d, 1)
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 1)
    with pytest.raises(ValueError, match="current device is cuda:1"):
        fsi.fsi_gamma_beta_noalloc(d.nx, d.ny, d.nz, d.lx, d.ly, d.lz, d.eta, x[:3 * d.nn], x[4 * d.nn:5 * d.nn], out)
