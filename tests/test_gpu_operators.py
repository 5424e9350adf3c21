"""GPU-vs-oracle parity of the element operators (residual, JVP, diagonal) and of
gamma/beta, through the C ABI.

FP64 tolerance: every operator is a fixed sum of O(100) float64 products per
quadrature point and node whose terms (gradients ~1/h, stabilisation, random
O(1) fields) can exceed the assembled entry by 10^2-10^3 through cancellation; the
CUDA path and the oracle order these sums differently, so entries agree to a few
hundred ulps of the largest term: max|gpu - oracle| <= 1e-10 * max|oracle|.
FP32 products (FSI_FP32): <= 2e-5 * max|oracle| (float32 unit roundoff 6e-8 times
the same O(100) terms, with cancellation headroom).
"""
import numpy as np
import pytest

from tests.gpu_helpers import Gpu, relmax

pytestmark = pytest.mark.gpu

from oracle import ac, blocks, cgt, diag, mobility, ns  # noqa: E402
from oracle.fields import Problem, State  # noqa: E402
from paper_2402_10348_gb300 import fsi  # noqa: E402
from tests.helpers import desc_small  # noqa: E402
from workloads import random_state  # noqa: E402

TOL64 = 1e-10
TOL32 = 2e-5

# sizes spanning several 15 x 15 node columns, z chunks and ragged tails
CASES = {
    "ragged": dict(n=(17, 19, 13), n_fluid=1, n_solid=1),
    "two_solids_rho_inf": dict(n=(9, 16, 7), n_fluid=2, n_solid=2, rho_inf=0.5, gravity=(0.0, -1.0, -9.81)),
    "single_element": dict(n=(1, 1, 1), n_fluid=1, n_solid=1),
    "no_solid_exact_tiles": dict(n=(14, 29, 4), n_fluid=1, n_solid=0, dirichlet=False),
    "four_solids": dict(n=(6, 5, 4), n_fluid=1, n_solid=4),
}


def _setup(case, seed=0):
    d = desc_small(**CASES[case])
    x1, xn, xdn = random_state(d, seed)
    return d, Problem(d), State(x1, xn, xdn), Gpu(d, x1, xn, xdn)


@pytest.mark.parametrize("case", list(CASES))
def test_ns_residual(case):
    d, pb, st, g = _setup(case)
    ref = ns.ns_residual(pb, st).ravel()
    got = g.residual(fsi.FSI_BLOCK_NS, 4 * d.nn)
    assert relmax(got, ref) <= TOL64


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("aug", [True, False])
def test_ns_jvp(case, aug):
    d, pb, st, g = _setup(case)
    dx = np.random.default_rng(1).normal(size=(4, d.nn))
    ref = ns.ns_jvp(pb, st, dx, elastic_aug=aug).ravel()
    got = g.jvp(fsi.FSI_BLOCK_NS, dx, fsi.FSI_ELASTIC_AUG if aug else 0)
    assert relmax(got, ref) <= TOL64
    got32 = g.jvp(fsi.FSI_BLOCK_NS, dx, (fsi.FSI_ELASTIC_AUG if aug else 0) | fsi.FSI_FP32)
    e32 = relmax(got32, ref)
    print(f"FP32 NS JVP {case} aug={aug}: max rel err {e32:.3e}")
    assert e32 <= TOL32


@pytest.mark.parametrize("case", ["ragged", "two_solids_rho_inf", "single_element"])
def test_ns_diagonal(case):
    d, pb, st, g = _setup(case)
    ref = diag.block_diagonal(pb, st, "ns")
    got = g.diag(fsi.FSI_BLOCK_NS, 4 * d.nn)
    assert relmax(got, ref) <= TOL64


@pytest.mark.parametrize("case", list(CASES))
def test_ac_operators(case):
    d, pb, st, g = _setup(case)
    for i in range(d.n_phase):
        gam, bet = 0.3 + 0.1 * i, -0.2 + 0.15 * i
        fsi.fsi_set_ac_coeffs(g.mesh, i, gam, bet)
        ref = ac.ac_residual(pb, st, i, gam, bet)
        assert relmax(g.residual(fsi.FSI_BLOCK_AC(i), d.nn), ref) <= TOL64
        dphi = np.random.default_rng(10 + i).normal(size=d.nn)
        ref = ac.ac_jvp(pb, st, i, gam, bet, dphi)
        assert relmax(g.jvp(fsi.FSI_BLOCK_AC(i), dphi), ref) <= TOL64
        assert relmax(g.jvp(fsi.FSI_BLOCK_AC(i), dphi, fsi.FSI_FP32), ref) <= TOL32
        if d.nn < 3000:
            coeffs = {"gamma": {i: gam}, "beta": {i: bet}}
            ref = diag.block_diagonal(pb, st, ("ac", i), coeffs)
            assert relmax(g.diag(fsi.FSI_BLOCK_AC(i), d.nn), ref) <= TOL64


@pytest.mark.parametrize("case", list(CASES))
def test_b_operators(case):
    d, pb, st, g = _setup(case)
    for s in range(d.n_solid):
        ref = cgt.cgt_residual(pb, st, s).ravel()
        assert relmax(g.residual(fsi.FSI_BLOCK_B(s), 6 * d.nn), ref) <= TOL64
        dB = np.random.default_rng(20 + s).normal(size=(6, d.nn))
        ref = cgt.cgt_jvp(pb, st, s, dB).ravel()
        assert relmax(g.jvp(fsi.FSI_BLOCK_B(s), dB), ref) <= TOL64
        assert relmax(g.jvp(fsi.FSI_BLOCK_B(s), dB, fsi.FSI_FP32), ref) <= TOL32
        if d.nn < 3000:
            ref = diag.block_diagonal(pb, st, ("b", s))
            assert relmax(g.diag(fsi.FSI_BLOCK_B(s), 6 * d.nn), ref) <= TOL64


@pytest.mark.parametrize("case", list(CASES))
def test_gamma_beta(case):
    d, pb, st, g = _setup(case)
    for i in range(d.n_phase):
        gam, bet = fsi.fsi_update_ac_coeffs(g.mesh, i, *g.st())
        assert gam == pytest.approx(mobility.mobility(pb, st, i), rel=1e-11, abs=1e-300)
        assert bet == pytest.approx(mobility.beta(pb, st, i), rel=1e-11, abs=1e-14)


def test_gamma_edge_cases():
    """No node in the band -> gamma = 0; fixed gamma overrides the model."""
    d = desc_small(n=(4, 4, 4), n_fluid=1, n_solid=0)
    x = np.zeros((d.ncomp, d.nn))
    x[0:3] = np.random.default_rng(0).normal(size=(3, d.nn))
    x[4] = 0.95
    g = Gpu(d, x, x, np.zeros_like(x))
    gam, bet = fsi.fsi_update_ac_coeffs(g.mesh, 0, *g.st())
    assert gam == 0.0
    assert bet == pytest.approx(2 * 0.95 * np.sign(0.95 ** 2 - 1), rel=1e-13)
    fsi.fsi_fix_gamma(g.mesh, 0, 0.7)
    gam, _ = fsi.fsi_update_ac_coeffs(g.mesh, 0, *g.st())
    assert gam == 0.7


def test_invalid_arguments_rejected():
    d = desc_small(n=(2, 2, 2))
    x1, xn, xdn = random_state(d, 0)
    g = Gpu(d, x1, xn, xdn)
    import torch
    r = torch.zeros(4 * d.nn, dtype=torch.float64, device="cuda:0")
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_residual(g.mesh, fsi.FSI_BLOCK_AC(7), *g.st(), r)
    assert e.value.code == fsi.FSI_EINVAL
    with pytest.raises(fsi.FsiError):
        fsi.fsi_residual(g.mesh, fsi.FSI_BLOCK_B(3), *g.st(), r)
    bad = desc_small(n=(2, 2, 2))
    bad.nx = 0
    with pytest.raises(fsi.FsiError):
        fsi.fsi_create_mesh(bad)


def test_ns_operators_with_independent_indicators():
    """Three phases whose fractions do not sum to one (each indicator its own sphere
    profile, as the indicators of N > 2 phases evolve independently): float64 residual
    and product against the oracle, float32 product within TOL32."""
    d = desc_small(n=(16, 13, 11), n_fluid=1, n_solid=2)
    x1, xn, xdn = random_state(d, 5, independent=True)
    alpha_sum = sum((1.0 + x1[4 + i]) / 2.0 for i in range(d.n_phase))
    assert np.abs(alpha_sum - 1.0).max() > 0.5  # not a partition of unity
    pb, st, g = Problem(d), State(x1, xn, xdn), Gpu(d, x1, xn, xdn)
    assert relmax(g.residual(fsi.FSI_BLOCK_NS, 4 * d.nn), ns.ns_residual(pb, st).ravel()) <= TOL64
    dx = np.random.default_rng(2).normal(size=(4, d.nn))
    ref = ns.ns_jvp(pb, st, dx).ravel()
    assert relmax(g.jvp(fsi.FSI_BLOCK_NS, dx), ref) <= TOL64
    assert relmax(g.jvp(fsi.FSI_BLOCK_NS, dx, fsi.FSI_ELASTIC_AUG | fsi.FSI_FP32), ref) <= TOL32
