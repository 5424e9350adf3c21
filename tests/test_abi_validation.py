"""Argument checks of the C ABI that run before any CUDA call (no GPU needed): bad mesh
descriptions, null handles and pointers, and the binding's refusal of host tensors."""
import ctypes as C
import threading

import pytest
import torch

from paper_2402_10348_gb300 import _build, fsi
from tests.helpers import desc_small


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def _create(d):
    s, ph = fsi.make_desc(d)
    h = C.c_void_p()
    rc = fsi.lib().fsi_create_mesh(C.byref(s), C.byref(h))
    return rc, fsi.lib().fsi_last_error().decode(), h


@pytest.mark.parametrize("change, words", [
    (dict(nx=0), "nx, ny, nz must be >= 1"),
    (dict(lz=-1.0), "box lengths must be > 0"),
    (dict(dt=0.0), "dt and eps must be > 0"),
    (dict(eps=-0.1), "dt and eps must be > 0"),
    (dict(rho_inf=1.5), "rho_inf must be in [0,1]"),
    (dict(pin_node=10 ** 6), "pin_node out of range"),
])
def test_bad_mesh_descriptions_are_rejected(change, words):
    d = desc_small(n=(3, 3, 3))
    for k, v in change.items():
        setattr(d, k, v)
    rc, msg, h = _create(d)
    assert rc == fsi.FSI_EINVAL and words in msg and not h.value


def test_bad_phases_are_rejected():
    d = desc_small(n=(3, 3, 3))
    d.phases[0].rho = 0.0
    rc, msg, _ = _create(d)
    assert rc == fsi.FSI_EINVAL and "rho > 0" in msg
    d = desc_small(n=(3, 3, 3), n_fluid=1, n_solid=16)  # 17 phases
    rc, msg, _ = _create(d)
    assert rc == fsi.FSI_EINVAL and "1..16 phases" in msg


def test_null_handles_and_pointers_are_rejected():
    L = fsi.lib()
    assert L.fsi_create_mesh(None, None) == fsi.FSI_EINVAL
    st = fsi.fsi_state()
    assert L.fsi_jvp(None, C.c_int32(0), C.byref(st), None, None, C.c_uint32(0)) == fsi.FSI_EINVAL
    assert L.fsi_residual(None, C.c_int32(0), C.byref(st), None) == fsi.FSI_EINVAL
    assert L.fsi_diag(None, C.c_int32(0), C.byref(st), None, C.c_uint32(0)) == fsi.FSI_EINVAL
    out = (C.c_double * 3)()
    assert L.fsi_center_of_mass(None, None, C.c_int32(0), out) == fsi.FSI_EINVAL
    assert L.fsi_track_points(None, None, C.c_int64(-1), None) == fsi.FSI_EINVAL


def test_last_error_is_per_thread():
    """A failing call in another thread leaves this thread's message alone."""
    d = desc_small(n=(3, 3, 3))
    d.dt = 0.0
    _create(d)
    mine = fsi.lib().fsi_last_error().decode()
    seen = []

    def other():
        d2 = desc_small(n=(3, 3, 3))
        d2.nx = 0
        seen.append(_create(d2)[1])

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert "nx, ny, nz" in seen[0]
    assert fsi.lib().fsi_last_error().decode() == mine


def test_binding_refuses_host_and_mistyped_tensors():
    with pytest.raises(ValueError, match="device"):
        fsi._ptr(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(TypeError, match="float64"):
        fsi._dptr(torch.zeros(4, dtype=torch.float32))
    with pytest.raises(TypeError):
        fsi._ptr([0.0, 1.0])


@pytest.mark.parametrize("which, sizes", [
    ("v", (3 * 5 * 5 * 5 - 1, 5 * 5 * 5, 2)),
    ("phi", (3 * 5 * 5 * 5, 5 * 5 * 5 - 1, 2)),
    ("gamma_beta", (3 * 5 * 5 * 5, 5 * 5 * 5, 1)),
])
def test_noalloc_binding_rejects_undersized_tensors(which, sizes):
    """fsi_gamma_beta_noalloc takes no mesh handle, so the binding checks the tensor
    sizes against the mesh sizes before anything reaches the library."""
    v, phi, gb = (torch.zeros(n, dtype=torch.float64) for n in sizes)
    with pytest.raises(ValueError, match=f"{which} has"):
        fsi.fsi_gamma_beta_noalloc(4, 4, 4, 1.0, 1.0, 1.0, 0.2, v, phi, gb)


def test_noalloc_binding_rejects_host_tensors():
    nn = 5 * 5 * 5
    v, phi, gb = (torch.zeros(n, dtype=torch.float64) for n in (3 * nn, nn, 2))
    with pytest.raises(ValueError, match="not a CUDA tensor"):
        fsi.fsi_gamma_beta_noalloc(4, 4, 4, 1.0, 1.0, 1.0, 0.2, v, phi, gb)
