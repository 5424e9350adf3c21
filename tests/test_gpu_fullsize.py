"""GPU-vs-oracle parity at the full workload sizes.

64^3 cavity (the benchmarked workload): whole residual / JVP vectors against the
oracle.  Falling sphere (96x96x192, 3 phases, 2 solids) and ship/ice (256x128x64,
11 phases, 9 solids): sampled outputs.  The operators are local (the result at a node
depends only on its 8 elements), so the oracle evaluates a 10^3-element window cut
out of the full-size state, and the GPU's full-size result is compared at the
window's strictly interior nodes.  Tolerances as in test_gpu_operators.
"""
import numpy as np
import pytest

from tests.gpu_helpers import DEV, Gpu, T, relmax

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from oracle import ac, cgt, mobility, ns  # noqa: E402
from oracle.fields import Problem, State  # noqa: E402
from paper_2402_10348_gb300 import fsi  # noqa: E402
from workloads import BC_NATURAL, FaceBC, cavity64, falling, random_state, shipice  # noqa: E402

TOL64 = 1e-10
TOL32 = 2e-5


@pytest.fixture(scope="module")
def cav():
    d = cavity64().desc
    x1, xn, xdn = random_state(d, 5)
    return d, Problem(d), State(x1, xn, xdn), Gpu(d, x1, xn, xdn)


def test_cavity64_ns_jvp_full_vector(cav):
    d, pb, st, g = cav
    dx = np.random.default_rng(2).normal(size=(4, d.nn))
    ref = ns.ns_jvp(pb, st, dx).ravel()
    assert relmax(g.jvp(fsi.FSI_BLOCK_NS, dx), ref) <= TOL64
    assert relmax(g.jvp(fsi.FSI_BLOCK_NS, dx, fsi.FSI_ELASTIC_AUG | fsi.FSI_FP32), ref) <= TOL32


def test_cavity64_residuals_full_vector(cav):
    d, pb, st, g = cav
    assert relmax(g.residual(fsi.FSI_BLOCK_NS, 4 * d.nn), ns.ns_residual(pb, st).ravel()) <= TOL64
    fsi.fsi_set_ac_coeffs(g.mesh, 1, 0.37, 0.11)
    assert relmax(g.residual(fsi.FSI_BLOCK_AC(1), d.nn), ac.ac_residual(pb, st, 1, 0.37, 0.11)) <= TOL64
    assert relmax(g.residual(fsi.FSI_BLOCK_B(0), 6 * d.nn), cgt.cgt_residual(pb, st, 0).ravel()) <= TOL64


def test_cavity64_gamma_beta(cav):
    d, pb, st, g = cav
    for i in range(d.n_phase):
        gam, bet = fsi.fsi_update_ac_coeffs(g.mesh, i, *g.st())
        assert gam == pytest.approx(mobility.mobility(pb, st, i), rel=1e-11)
        assert bet == pytest.approx(mobility.beta(pb, st, i), rel=1e-11)


# ------------------------------------------------------------- sampled windows
def _window(desc, states, corner, size):
    """Sub-problem of `size` elements starting at element `corner`, natural
    boundaries (no Dirichlet rows), same spacing; and the node map into the full mesh."""
    import copy
    sub = copy.deepcopy(desc)
    hx, hy, hz = desc.h
    sub.nx, sub.ny, sub.nz = size
    sub.lx, sub.ly, sub.lz = size[0] * hx, size[1] * hy, size[2] * hz
    sub.faces = [FaceBC(BC_NATURAL) for _ in range(6)]
    sub.prescribed_box = None
    sub.pin_node = -1
    i0, j0, k0 = corner
    ii, jj, kk = np.meshgrid(np.arange(size[0] + 1) + i0, np.arange(size[1] + 1) + j0,
                             np.arange(size[2] + 1) + k0, indexing="ij")
    ii, jj, kk = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, kk))
    nodes = ii + (desc.nx + 1) * (jj + (desc.ny + 1) * kk)
    li, lj, lk = (np.arange(sub.nn) % (size[0] + 1), (np.arange(sub.nn) // (size[0] + 1)) % (size[1] + 1),
                  np.arange(sub.nn) // ((size[0] + 1) * (size[1] + 1)))
    inner = (li > 0) & (li < size[0]) & (lj > 0) & (lj < size[1]) & (lk > 0) & (lk < size[2])
    return sub, [s[:, nodes] for s in states], nodes, inner


@pytest.mark.parametrize("wl_name", ["falling", "shipice"])
def test_large_workloads_sampled_windows(wl_name):
    wl = falling() if wl_name == "falling" else shipice()
    d = wl.desc
    x1, xn, xdn = random_state(d, 9, noise=0.02)
    g = Gpu(d, x1, xn, xdn)
    rng = np.random.default_rng(4)
    size = (10, 10, 10)
    dx_full = rng.normal(size=(d.ncomp, d.nn))
    out = {}
    out["ns_jvp"] = g.jvp(fsi.FSI_BLOCK_NS, dx_full[0:4]).reshape(4, d.nn)
    out["ns_jvp32"] = g.jvp(fsi.FSI_BLOCK_NS, dx_full[0:4], fsi.FSI_ELASTIC_AUG | fsi.FSI_FP32).reshape(4, d.nn)
    out["ns_res"] = g.residual(fsi.FSI_BLOCK_NS, 4 * d.nn).reshape(4, d.nn)
    i_ac = d.n_phase - 1
    fsi.fsi_set_ac_coeffs(g.mesh, i_ac, 0.5, 0.2)
    out["ac_jvp"] = g.jvp(fsi.FSI_BLOCK_AC(i_ac), dx_full[4 + i_ac])
    s_b = d.n_solid - 1
    b0 = 4 + d.n_phase + 6 * s_b
    out["b_jvp"] = g.jvp(fsi.FSI_BLOCK_B(s_b), dx_full[b0:b0 + 6]).reshape(6, d.nn)
    for w in range(3):
        corner = tuple(int(rng.integers(1, n - size[k] - 1)) for k, n in enumerate((d.nx, d.ny, d.nz)))
        sub, (s1, sn, sd), nodes, inner = _window(d, (x1, xn, xdn), corner, size)
        pb, st = Problem(sub), State(s1, sn, sd)
        ddx = dx_full[:, nodes]
        ref = ns.ns_jvp(pb, st, ddx[0:4])
        assert relmax(out["ns_jvp"][:, nodes][:, inner], ref[:, inner]) <= TOL64, (wl_name, w)
        assert relmax(out["ns_jvp32"][:, nodes][:, inner], ref[:, inner]) <= TOL32, (wl_name, w)
        ref = ns.ns_residual(pb, st)
        assert relmax(out["ns_res"][:, nodes][:, inner], ref[:, inner]) <= TOL64, (wl_name, w)
        ref = ac.ac_jvp(pb, st, i_ac, 0.5, 0.2, ddx[4 + i_ac])
        assert relmax(out["ac_jvp"][nodes][inner], ref[inner]) <= TOL64, (wl_name, w)
        ref = cgt.cgt_jvp(pb, st, s_b, ddx[b0:b0 + 6])
        assert relmax(out["b_jvp"][:, nodes][:, inner], ref[:, inner]) <= TOL64, (wl_name, w)


def test_cavity64_init_tags_sampled():
    """Grid-cell tags at full size, bit-exact at 3000 sampled nodes."""
    from oracle.gridcell import signed_distance_phi
    wl = cavity64()
    d = wl.desc
    g = Gpu(d, *random_state(d, 0))
    phi = torch.zeros(d.n_phase * d.nn, dtype=torch.float64, device=DEV)
    tags = torch.zeros(4 * d.nn, dtype=torch.int32, device=DEV)
    fsi.fsi_init_phases(g.mesh, wl.surfaces, wl.rules, wl.grid_cells, phi, tags)
    torch.cuda.synchronize()
    nodes = np.random.default_rng(3).choice(d.nn, 3000, replace=False)
    ref_phi, ref_tags = signed_distance_phi(d, wl.surfaces[0], d.eps, wl.grid_cells, nodes=nodes)
    got = tags.cpu().numpy().reshape(4, d.nn)
    assert np.array_equal(got[:, nodes], ref_tags[:, nodes])
    gp = phi.cpu().numpy().reshape(d.n_phase, d.nn)
    assert np.abs(gp[1, nodes] - ref_phi[nodes]).max() <= 4e-16
