"""Python binding of libfsi (include/fsi.h): argument marshalling only.

Every function has the name of the C entry point it calls and forwards device
pointers of torch CUDA tensors; all computation happens in libfsi's kernels.  A
missing library raises immediately: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsi.so")

FSI_OK, FSI_EINVAL, FSI_ECUDA, FSI_ENOCONV, FSI_ENAN, FSI_ETIMEOUT, FSI_ENOMEM = range(7)
FSI_BLOCK_NS = 0
FSI_ELASTIC_AUG = 0x1
FSI_FP32 = 0x2
FSI_PC_NONE, FSI_PC_JACOBI, FSI_PC_LEARNED = 0, 1, 2
FSI_HARVEST = 0x10
FSI_PC_ALTERNATE = 0x20
FSI_NO_STALL_STOP = 0x40
FSI_PINNED_SOLVE = 0x80
FSI_PREC_FP64, FSI_PREC_FP32_IR = 0, 1
FSI_BC_NATURAL, FSI_BC_DIRICHLET = 0, 1
FSI_RULE_SURFACE, FSI_RULE_COMPLEMENT = 0, 1


def FSI_BLOCK_AC(i: int) -> int:
    return 0x10000 | i


def FSI_BLOCK_B(s: int) -> int:
    return 0x20000 | s


class FsiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfsi error {code}: {msg}")
        self.code = code


class fsi_phase(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("mu_L", C.c_double),
                ("is_solid", C.c_int32), ("pad", C.c_int32)]


class fsi_face_bc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("priority", C.c_int32), ("vel", C.c_double * 3)]


class fsi_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_phase", C.c_int32),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("phases", C.POINTER(fsi_phase)),
                ("gravity", C.c_double * 3),
                ("eps", C.c_double), ("eta", C.c_double), ("dt", C.c_double),
                ("rho_inf", C.c_double), ("c_i", C.c_double),
                ("faces", fsi_face_bc * 6),
                ("has_box", C.c_int32), ("pin_node", C.c_int32),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("box_vel", C.c_double * 3),
                ("device", C.c_int32), ("pad", C.c_int32)]


class fsi_state(C.Structure):
    _fields_ = [("x", C.c_void_p), ("xn", C.c_void_p), ("xdn", C.c_void_p)]


class fsi_solve_opts(C.Structure):
    _fields_ = [("m", C.c_int32), ("max_iter", C.c_int32), ("rtol", C.c_double),
                ("precond", C.c_int32), ("precision", C.c_int32), ("flags", C.c_uint32),
                ("ir_max", C.c_int32), ("ir_inner_rtol", C.c_double)]


class fsi_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("refinements", C.c_int32),
                ("applies", C.c_int32), ("rel_res", C.c_double), ("stalled", C.c_int32), ("fallback", C.c_int32)]


class fsi_step_opts(C.Structure):
    _fields_ = [("k_max", C.c_int32), ("fixed_iters", C.c_int32), ("nl_tol", C.c_double),
                ("solve", fsi_solve_opts)]


class fsi_step_info(C.Structure):
    _fields_ = [("nl_iters", C.c_int32), ("gmres_iters_ns", C.c_int32), ("gmres_iters_ac", C.c_int32),
                ("gmres_iters_b", C.c_int32), ("applies", C.c_int32), ("stalled_solves", C.c_int32),
                ("dof_applied", C.c_int64), ("max_ratio", C.c_double), ("worst_rel_res", C.c_double),
                ("fallback_solves", C.c_int32), ("pad", C.c_int32)]


class fsi_surface(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("tris", C.c_void_p), ("n_verts", C.c_int32), ("n_tris", C.c_int32)]


class fsi_phase_rule(C.Structure):
    _fields_ = [("kind", C.c_int32), ("surface", C.c_int32), ("plane_z", C.c_double),
                ("plane_side", C.c_int32), ("pad", C.c_int32)]


class fsi_profile_entry(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("ms", C.c_double), ("bytes", C.c_double)]


FSI_PROF_CLASSES = 26

EXPORTS = ["fsi_create_mesh", "fsi_destroy_mesh", "fsi_set_stream", "fsi_mesh_info", "fsi_residual",
           "fsi_jvp", "fsi_diag", "fsi_update_ac_coeffs", "fsi_set_ac_coeffs", "fsi_fix_gamma",
           "fsi_set_pressure_pin",
           "fsi_gmres", "fsi_step", "fsi_init_phases", "fsi_gamma_beta_noalloc", "fsi_profile",
           "fsi_profile_read", "fsi_pc_create", "fsi_pc_destroy", "fsi_pc_layout", "fsi_pc_set_weights",
           "fsi_pc_get_weights", "fsi_pc_set_norm", "fsi_pc_get_norm", "fsi_pc_forward", "fsi_pc_grad",
           "fsi_pc_apply", "fsi_pc_add_pair", "fsi_pc_add_smooth_pairs", "fsi_pc_pairs", "fsi_pc_fit_norm", "fsi_pc_train", "fsi_set_pc",
           "fsi_batch_create", "fsi_batch_destroy", "fsi_batch_layout", "fsi_batch_jvp", "fsi_batch_gmres",
           "fsi_batch_autotune", "fsi_batch_set_graph", "fsi_center_of_mass", "fsi_track_points",
           "fsi_probe_peaks", "fsi_batch_create_blocks", "fsi_batch_stepper_create", "fsi_batch_stepper_destroy",
           "fsi_batch_step", "fsi_create_tet_mesh", "fsi_last_error"]

_lib = None


def lib():
    """Loads libfsi.so (built in-tree by paper_2402_10348_gb300._build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        L.fsi_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name != "fsi_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int, allow=()):
    if rc != FSI_OK and rc not in allow:
        raise FsiError(rc, lib().fsi_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("libfsi takes device (CUDA) tensors")
    if not t.is_contiguous():
        raise ValueError("libfsi takes contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _dptr(t):
    if t.dtype != torch.float64:
        raise TypeError("libfsi field arrays are float64")
    return _ptr(t)


class Mesh:
    """Owns an fsi_mesh handle."""

    def __init__(self, handle, desc_struct, phases_arr):
        self.handle = handle
        self._desc = desc_struct
        self._phases = phases_arr
        nc, nn, ns = C.c_int32(), C.c_int64(), C.c_int32()
        _check(lib().fsi_mesh_info(handle, C.byref(nc), C.byref(nn), C.byref(ns)))
        self.ncomp, self.nn, self.n_solid = nc.value, nn.value, ns.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.fsi_destroy_mesh(h)
            self.handle = None


def make_desc(d, device: int = 0):
    """fsi_mesh_desc from a problem description with the fields of workloads.MeshDesc."""
    ph = (fsi_phase * len(d.phases))()
    for i, p in enumerate(d.phases):
        ph[i] = fsi_phase(p.rho, p.mu, p.mu_L, 1 if p.solid else 0, 0)
    s = fsi_mesh_desc()
    s.nx, s.ny, s.nz, s.n_phase = d.nx, d.ny, d.nz, len(d.phases)
    s.lx, s.ly, s.lz = d.lx, d.ly, d.lz
    s.phases = C.cast(ph, C.POINTER(fsi_phase))
    s.gravity[:] = list(d.gravity)
    s.eps, s.eta, s.dt, s.rho_inf, s.c_i = d.eps, d.eta, d.dt, d.rho_inf, d.c_i
    for f in range(6):
        fb = d.faces[f]
        s.faces[f].kind, s.faces[f].priority = fb.kind, fb.priority
        s.faces[f].vel[:] = list(fb.vel)
    if d.prescribed_box is not None:
        lo, hi, vel = d.prescribed_box
        s.has_box = 1
        s.box_lo[:], s.box_hi[:], s.box_vel[:] = list(lo), list(hi), list(vel)
    s.pin_node = d.pin_node
    s.device = device
    return s, ph


def fsi_create_mesh(d, device: int = 0) -> Mesh:
    s, ph = make_desc(d, device)
    h = C.c_void_p()
    _check(lib().fsi_create_mesh(C.byref(s), C.byref(h)))
    return Mesh(h, s, ph)


def fsi_create_tet_mesh(d, coords, conn, device: int = 0) -> Mesh:
    """A linear-tetrahedron mesh on the nodes of d's box grid: coords host float64 [3, nn],
    conn host int [ne, 4] (positively oriented)."""
    import numpy as np
    s, ph = make_desc(d, device)
    X = np.ascontiguousarray(coords, dtype=np.float64)
    T = np.ascontiguousarray(conn, dtype=np.int32)
    if X.shape != (3, d.nn) or T.ndim != 2 or T.shape[1] != 4:
        raise ValueError("coords must be [3, nn] and conn [ne, 4]")
    h = C.c_void_p()
    _check(lib().fsi_create_tet_mesh(C.byref(s), X.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p),
                                     C.c_int64(T.shape[0]), C.byref(h)))
    return Mesh(h, s, ph)


def fsi_set_stream(mesh: Mesh, stream=None):
    st = torch.cuda.current_stream() if stream is None else stream
    _check(lib().fsi_set_stream(mesh.handle, C.c_void_p(st.cuda_stream)))


def _state(x, xn, xdn):
    return fsi_state(_dptr(x), _dptr(xn), _dptr(xdn))


def fsi_residual(mesh: Mesh, block: int, x, xn, xdn, r):
    st = _state(x, xn, xdn)
    _check(lib().fsi_residual(mesh.handle, C.c_int32(block), C.byref(st), _dptr(r)))


def fsi_jvp(mesh: Mesh, block: int, x, xn, xdn, dx, y, flags: int = FSI_ELASTIC_AUG):
    st = _state(x, xn, xdn)
    _check(lib().fsi_jvp(mesh.handle, C.c_int32(block), C.byref(st), _dptr(dx), _dptr(y), C.c_uint32(flags)))


def fsi_diag(mesh: Mesh, block: int, x, xn, xdn, d, flags: int = FSI_ELASTIC_AUG):
    st = _state(x, xn, xdn)
    _check(lib().fsi_diag(mesh.handle, C.c_int32(block), C.byref(st), _dptr(d), C.c_uint32(flags)))


def fsi_update_ac_coeffs(mesh: Mesh, phase: int, x, xn, xdn):
    st = _state(x, xn, xdn)
    out = (C.c_double * 2)()
    _check(lib().fsi_update_ac_coeffs(mesh.handle, C.c_int32(phase), C.byref(st), out))
    return out[0], out[1]


def fsi_set_ac_coeffs(mesh: Mesh, phase: int, gamma: float, beta: float):
    _check(lib().fsi_set_ac_coeffs(mesh.handle, C.c_int32(phase), C.c_double(gamma), C.c_double(beta)))


def fsi_fix_gamma(mesh: Mesh, phase: int, gamma: float):
    _check(lib().fsi_fix_gamma(mesh.handle, C.c_int32(phase), C.c_double(gamma)))


def fsi_set_pressure_pin(mesh: Mesh, active: bool):
    _check(lib().fsi_set_pressure_pin(mesh.handle, C.c_int32(1 if active else 0)))


def solve_opts(m=30, max_iter=2000, rtol=1e-8, precond=FSI_PC_JACOBI, precision=FSI_PREC_FP64,
               flags=FSI_ELASTIC_AUG, ir_max=10, ir_inner_rtol=1e-3) -> fsi_solve_opts:
    return fsi_solve_opts(m, max_iter, rtol, precond, precision, flags, ir_max, ir_inner_rtol)


def fsi_gmres(mesh: Mesh, block: int, x, xn, xdn, rhs, sol, opts: fsi_solve_opts, allow_noconv=False):
    st = _state(x, xn, xdn)
    info = fsi_solve_info()
    _check(lib().fsi_gmres(mesh.handle, C.c_int32(block), C.byref(st), _dptr(rhs), _dptr(sol),
                           C.byref(opts), C.byref(info)), allow=(FSI_ENOCONV,) if allow_noconv else ())
    return info


def fsi_step(mesh: Mesh, x, xn, xdn, k_max=5, nl_tol=5e-4, fixed_iters=False,
             solve: fsi_solve_opts | None = None) -> fsi_step_info:
    st = _state(x, xn, xdn)
    o = fsi_step_opts(k_max, 1 if fixed_iters else 0, nl_tol, solve if solve is not None else solve_opts())
    info = fsi_step_info()
    _check(lib().fsi_step(mesh.handle, C.byref(st), C.byref(o), C.byref(info)))
    return info


def fsi_init_phases(mesh: Mesh, surfaces, rules, grid, phi_out, tags_out=None):
    """surfaces: objects with .verts (n,3) float64 and .tris (m,3) int arrays (host);
    rules: objects with kind, surface, plane_z, plane_side."""
    import numpy as np
    keep = []
    S = (fsi_surface * max(1, len(surfaces)))()
    for i, s in enumerate(surfaces):
        v = np.ascontiguousarray(s.verts, dtype=np.float64)
        t = np.ascontiguousarray(s.tris, dtype=np.int32)
        keep += [v, t]
        S[i] = fsi_surface(v.ctypes.data, t.ctypes.data, v.shape[0], t.shape[0])
    R = (fsi_phase_rule * len(rules))()
    for i, r in enumerate(rules):
        R[i] = fsi_phase_rule(r.kind, r.surface, r.plane_z, r.plane_side, 0)
    tp = None
    if tags_out is not None:
        if tags_out.dtype != torch.int32:
            raise TypeError("tags are int32")
        tp = _ptr(tags_out)
    _check(lib().fsi_init_phases(mesh.handle, S, C.c_int32(len(surfaces)), R, C.c_int32(grid[0]),
                                 C.c_int32(grid[1]), C.c_int32(grid[2]), _dptr(phi_out), tp))


def fsi_center_of_mass(mesh: Mesh, x, solid: int):
    """(x, y, z) centre of mass of solid `solid` from the device state x; synchronises."""
    out = (C.c_double * 3)()
    _check(lib().fsi_center_of_mass(mesh.handle, _dptr(x), C.c_int32(solid), out))
    return out[0], out[1], out[2]


def fsi_track_points(mesh: Mesh, x, points):
    """Moves the device float64 points [n, 3] in place by one step with the velocity of x."""
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points: a [n, 3] tensor")
    n = points.shape[0]
    _check(lib().fsi_track_points(mesh.handle, _dptr(x), C.c_int64(n), _dptr(points) if n else None))


def fsi_gamma_beta_noalloc(nx, ny, nz, lx, ly, lz, eta, v, phi, gamma_beta, stream=None):
    """gamma, beta of one phase written to the device tensor gamma_beta[2]; no allocation.
    v: device float64 [3*nn] (v^{n+alpha}), phi: device float64 [nn] (phi^{n+alpha}),
    nn = (nx+1)(ny+1)(nz+1).  The C call takes no mesh handle, so the sizes and the
    device are checked here: undersized tensors or tensors on a GPU other than the
    current one raise ValueError before anything is launched."""
    for name, t in (("v", v), ("phi", phi), ("gamma_beta", gamma_beta)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name}: expected a torch tensor")
    if min(nx, ny, nz) >= 1:
        nn = (nx + 1) * (ny + 1) * (nz + 1)
        for name, t, need in (("v", v, 3 * nn), ("phi", phi, nn), ("gamma_beta", gamma_beta, 2)):
            if t.numel() < need:
                raise ValueError(f"fsi_gamma_beta_noalloc: {name} has {t.numel()} elements, needs {need}")
    for name, t in (("v", v), ("phi", phi), ("gamma_beta", gamma_beta)):
        if not t.is_cuda:
            raise ValueError(f"fsi_gamma_beta_noalloc: {name} is not a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"fsi_gamma_beta_noalloc: {name} is on cuda:{t.device.index}, "
                             f"the current device is cuda:{torch.cuda.current_device()}")
    st = torch.cuda.current_stream() if stream is None else stream
    _check(lib().fsi_gamma_beta_noalloc(C.c_int32(nx), C.c_int32(ny), C.c_int32(nz), C.c_double(lx),
                                        C.c_double(ly), C.c_double(lz), C.c_double(eta), _dptr(v), _dptr(phi),
                                        _dptr(gamma_beta), C.c_void_p(st.cuda_stream)))


def fsi_probe_peaks() -> dict:
    """Measured float32/float64 FMA rates (TFLOP/s) and read/copy bandwidth (GB/s)."""
    v = [C.c_double() for _ in range(4)]
    _check(lib().fsi_probe_peaks(*[C.byref(x) for x in v]))
    return {"fp32_tflops": v[0].value, "fp64_tflops": v[1].value, "read_gbs": v[2].value, "copy_gbs": v[3].value}


def fsi_profile(mesh: Mesh, enable: bool):
    _check(lib().fsi_profile(mesh.handle, C.c_int32(1 if enable else 0)))


def fsi_profile_read(mesh: Mesh) -> dict:
    """{kernel class: (launches, summed event ms)}; synchronises the mesh's stream."""
    out = (fsi_profile_entry * FSI_PROF_CLASSES)()
    n = C.c_int32()
    _check(lib().fsi_profile_read(mesh.handle, out, C.byref(n)))
    return {out[i].name.decode(): (out[i].launches, out[i].ms, out[i].bytes) for i in range(n.value)}


# ------------------------------------------------------------------ learned preconditioner
class fsi_pc_desc(C.Structure):
    _fields_ = [("block", C.c_int32), ("n_pairs_cap", C.c_int32), ("linear", C.c_int32), ("modulate", C.c_int32),
                ("smooth", C.c_int32), ("pad", C.c_int32)]


class PC:
    """Owns an fsi_pc handle; keeps its mesh alive."""

    def __init__(self, handle, mesh: Mesh):
        self.handle = handle
        self.mesh = mesh
        nl, nw = C.c_int32(), C.c_int64()
        fan = (C.c_int32 * 30)()
        grids = (C.c_int32 * 12)()
        _check(lib().fsi_pc_layout(handle, C.byref(nl), C.byref(nw), fan, grids))
        self.n_weights = nw.value
        self.fan = [(fan[2 * i], fan[2 * i + 1]) for i in range(nl.value)]
        self.grids = [(grids[3 * i], grids[3 * i + 1], grids[3 * i + 2]) for i in range(4)]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.fsi_pc_destroy(h)
            self.handle = None


def fsi_pc_create(mesh: Mesh, block: int = 0, n_pairs_cap: int = 0, linear: bool = False,
                  modulate: bool = False, smooth: bool = False) -> PC:
    h = C.c_void_p()
    d = fsi_pc_desc(block, n_pairs_cap, 1 if linear else 0, 1 if modulate else 0, 1 if smooth else 0, 0)
    _check(lib().fsi_pc_create(mesh.handle, C.byref(d), C.byref(h)))
    return PC(h, mesh)


def _f32_host(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def fsi_pc_set_weights(pc: PC, w):
    a, p = _f32_host(w)
    _check(lib().fsi_pc_set_weights(pc.handle, p, C.c_int64(a.size)))


def fsi_pc_get_weights(pc: PC):
    import numpy as np
    a = np.zeros(pc.n_weights, dtype=np.float32)
    _check(lib().fsi_pc_get_weights(pc.handle, a.ctypes.data_as(C.POINTER(C.c_float)), C.c_int64(a.size)))
    return a


def fsi_pc_set_norm(pc: PC, dbar, kc):
    d = (C.c_double * 4)(*[float(v) for v in dbar])
    k = (C.c_double * 4)(*[float(v) for v in kc])
    _check(lib().fsi_pc_set_norm(pc.handle, d, k))


def fsi_pc_get_norm(pc: PC):
    d, k = (C.c_double * 4)(), (C.c_double * 4)()
    _check(lib().fsi_pc_get_norm(pc.handle, d, k))
    return list(d), list(k)


def fsi_pc_forward(pc: PC, x_in, y):
    """x_in: device int16 tensor holding the bfloat16 input planes; y: float32 [4][nn]."""
    if x_in.dtype not in (torch.int16, torch.bfloat16) or y.dtype != torch.float32:
        raise TypeError("fsi_pc_forward: x_in is bfloat16 (or its int16 bits), y float32")
    _check(lib().fsi_pc_forward(pc.handle, _ptr(x_in), _ptr(y)))


def fsi_pc_grad(pc: PC, x_in, target, grad) -> float:
    if grad.dtype != torch.float32:
        raise TypeError("fsi_pc_grad: grad is float32")
    loss = C.c_double()
    _check(lib().fsi_pc_grad(pc.handle, _ptr(x_in), _ptr(target), _ptr(grad), C.byref(loss)))
    return loss.value


def fsi_pc_apply(pc: PC, x, xn, xdn, r, z):
    st = _state(x, xn, xdn)
    _check(lib().fsi_pc_apply(pc.handle, C.byref(st), _dptr(r), _dptr(z)))


def fsi_pc_add_pair(pc: PC, x, xn, xdn, r, e):
    st = _state(x, xn, xdn)
    _check(lib().fsi_pc_add_pair(pc.handle, C.byref(st), _dptr(r), _dptr(e)))


def fsi_pc_add_smooth_pairs(pc: PC, x, xn, xdn, count: int, seed: int = 0):
    st = _state(x, xn, xdn)
    _check(lib().fsi_pc_add_smooth_pairs(pc.handle, C.byref(st), C.c_int32(count), C.c_uint64(seed)))


def fsi_pc_pairs(pc: PC) -> int:
    n = C.c_int32()
    _check(lib().fsi_pc_pairs(pc.handle, C.byref(n)))
    return n.value


def fsi_pc_fit_norm(pc: PC):
    _check(lib().fsi_pc_fit_norm(pc.handle))


def fsi_pc_train(pc: PC, order, lr: float):
    """Adam steps over the stored pairs order[0..]; returns the loss before each step."""
    import numpy as np
    o = np.ascontiguousarray(order, dtype=np.int32)
    loss = np.zeros(o.size, dtype=np.float32)
    _check(lib().fsi_pc_train(pc.handle, C.c_int32(o.size), C.c_float(lr),
                              o.ctypes.data_as(C.POINTER(C.c_int32)),
                              loss.ctypes.data_as(C.POINTER(C.c_float))))
    return loss


def fsi_set_pc(mesh: Mesh, pc):
    _check(lib().fsi_set_pc(mesh.handle, pc.handle if pc is not None else None))


# ------------------------------------------------------------------ batched instances
class Batch:
    """Owns an fsi_batch handle; keeps its meshes alive."""

    def __init__(self, handle, meshes):
        self.handle = handle
        self.meshes = list(meshes)
        self.n = len(self.meshes)
        off = (C.c_int64 * (self.n + 1))()
        _check(lib().fsi_batch_layout(handle, off, None, None, None))
        self.offsets = [off[i] for i in range(self.n + 1)]

    def layout(self):
        tm, gm, la = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib().fsi_batch_layout(self.handle, None, C.byref(tm), C.byref(gm), C.byref(la)))
        return tm.value, gm.value, la.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.fsi_batch_destroy(h)
            self.handle = None


def _states(states):
    arr = (fsi_state * len(states))()
    for i, (x, xn, xdn) in enumerate(states):
        arr[i] = _state(x, xn, xdn)
    return arr


def fsi_batch_create(meshes, block: int = 0, m: int = 64) -> Batch:
    arr = (C.c_void_p * len(meshes))(*[mm.handle.value if hasattr(mm.handle, "value") else mm.handle
                                       for mm in meshes])
    h = C.c_void_p()
    _check(lib().fsi_batch_create(arr, C.c_int32(len(meshes)), C.c_int32(block), C.c_int32(m), C.byref(h)))
    return Batch(h, meshes)


def fsi_batch_create_blocks(meshes, blocks, m: int = 64) -> Batch:
    """A batch whose entry i solves block blocks[i] of meshes[i] (a mesh may repeat)."""
    arr = (C.c_void_p * len(meshes))(*[mm.handle.value if hasattr(mm.handle, "value") else mm.handle
                                       for mm in meshes])
    blk = (C.c_int32 * len(blocks))(*blocks)
    h = C.c_void_p()
    _check(lib().fsi_batch_create_blocks(arr, blk, C.c_int32(len(meshes)), C.c_int32(m), C.byref(h)))
    return Batch(h, meshes)


class BatchStepper:
    """Owns an fsi_batch_stepper handle; keeps its meshes alive."""

    def __init__(self, handle, meshes, m):
        self.handle = handle
        self.meshes = list(meshes)
        self.n = len(self.meshes)
        self.m = m

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.fsi_batch_stepper_destroy(h)
            self.handle = None


def fsi_batch_stepper_create(meshes, m: int = 30) -> BatchStepper:
    arr = (C.c_void_p * len(meshes))(*[mm.handle.value if hasattr(mm.handle, "value") else mm.handle
                                       for mm in meshes])
    h = C.c_void_p()
    _check(lib().fsi_batch_stepper_create(arr, C.c_int32(len(meshes)), C.c_int32(m), C.byref(h)))
    return BatchStepper(h, meshes, m)


def fsi_batch_step(stepper: BatchStepper, states, k_max=5, nl_tol=5e-4, fixed_iters=False,
                   solve: fsi_solve_opts | None = None):
    """One batched time step of every instance; states: list of (x, xn, xdn) device
    tensors advanced in place.  Returns the per-instance fsi_step_info list."""
    st = _states(states)
    o = fsi_step_opts(k_max, 1 if fixed_iters else 0, nl_tol,
                      solve if solve is not None else solve_opts(m=stepper.m))
    infos = (fsi_step_info * stepper.n)()
    _check(lib().fsi_batch_step(stepper.handle, st, C.byref(o), infos))
    return list(infos)


def fsi_batch_jvp(batch: Batch, states, dx, y, flags: int = FSI_ELASTIC_AUG):
    st = _states(states)
    _check(lib().fsi_batch_jvp(batch.handle, st, _dptr(dx), _dptr(y), C.c_uint32(flags)))


def fsi_batch_gmres(batch: Batch, states, rhs, sol, opts: fsi_solve_opts, allow_noconv=False):
    st = _states(states)
    infos = (fsi_solve_info * batch.n)()
    _check(lib().fsi_batch_gmres(batch.handle, st, _dptr(rhs), _dptr(sol), C.byref(opts), infos),
           allow=(FSI_ENOCONV,) if allow_noconv else ())
    return list(infos)


def fsi_batch_autotune(batch: Batch, states, flags: int = FSI_ELASTIC_AUG | FSI_FP32):
    st = _states(states)
    tm, gm, us = C.c_int32(), C.c_int32(), C.c_double()
    _check(lib().fsi_batch_autotune(batch.handle, st, C.c_uint32(flags), C.byref(tm), C.byref(gm), C.byref(us)))
    return tm.value, gm.value, us.value


def fsi_batch_set_graph(batch: Batch, use_graph: bool):
    _check(lib().fsi_batch_set_graph(batch.handle, C.c_int32(1 if use_graph else 0)))
