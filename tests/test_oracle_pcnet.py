"""Pins of the learned-preconditioner oracle (oracle/pcnet.py) and of FGMRES.

Each pin comes from outside the code under test: brute-force loops, adjoint
identities, closed forms (Q1 interpolation reproduces linear fields, full weighting
of a constant), finite differences, the closed form of Adam's first steps, torch's
own bfloat16 rounding, and dense linear algebra."""
import numpy as np
import pytest
import torch

from oracle import gmres as og
from oracle import pcnet as pn
from workloads import he_normal_weights


def _rng(s=0):
    return np.random.default_rng(s)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    x = _rng().normal(size=20000) * 10.0 ** _rng(1).integers(-30, 30, size=20000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(pn.bf16(x), ref)
    assert pn.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0            # tie -> even (down)
    assert pn.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6  # tie -> even (up)


def test_conv3_brute_force():
    x = _rng().normal(size=(2, 3, 4, 5))
    W = _rng(1).normal(size=(3, 2, 3, 3, 3))
    ref = np.zeros((3, 3, 4, 5))
    for o in range(3):
        for z in range(3):
            for y in range(4):
                for xx in range(5):
                    s = 0.0
                    for i in range(2):
                        for kz in range(3):
                            for ky in range(3):
                                for kx in range(3):
                                    zz, yy, xi = z + kz - 1, y + ky - 1, xx + kx - 1
                                    if 0 <= zz < 3 and 0 <= yy < 4 and 0 <= xi < 5:
                                        s += W[o, i, kz, ky, kx] * x[i, zz, yy, xi]
                    ref[o, z, y, xx] = s
    assert np.allclose(pn.conv3(x, W), ref, rtol=1e-13, atol=1e-13)


def test_conv3_adjoint_and_wgrad_identities():
    x = _rng().normal(size=(3, 4, 5, 6))
    W = _rng(1).normal(size=(2, 3, 3, 3, 3))
    g = _rng(2).normal(size=(2, 4, 5, 6))
    lhs = float((pn.conv3(x, W) * g).sum())
    assert lhs == pytest.approx(float((x * pn.conv3_adjoint(g, W)).sum()), rel=1e-12)
    # <g, conv3(x, W)> is linear in W with gradient conv3_wgrad(x, g)
    assert lhs == pytest.approx(float((pn.conv3_wgrad(x, g) * W).sum()), rel=1e-12)
    # one entry by brute force: dW[o, i, kz, ky, kx]
    o, i, kz, ky, kx = 1, 2, 0, 2, 1
    s = 0.0
    for z in range(4):
        for y in range(5):
            for xx in range(6):
                zz, yy, xi = z + kz - 1, y + ky - 1, xx + kx - 1
                if 0 <= zz < 4 and 0 <= yy < 5 and 0 <= xi < 6:
                    s += g[o, z, y, xx] * x[i, zz, yy, xi]
    assert pn.conv3_wgrad(x, g)[o, i, kz, ky, kx] == pytest.approx(s, rel=1e-12)


def test_level_shapes():
    assert pn.level_shapes((65, 65, 65)) == [(65,) * 3, (33,) * 3, (17,) * 3, (9,) * 3]
    assert pn.level_shapes((193, 97, 97))[-1] == (25, 13, 13)
    assert pn.level_shapes((8, 7, 9))[1] == (5, 4, 5)


@pytest.mark.parametrize("fine", [(9, 7, 5), (8, 6, 4)])
def test_prolongation_reproduces_linear_fields(fine):
    coarse = tuple(n // 2 + 1 for n in fine)
    a, b = 0.3, np.array([0.7, -1.1, 2.3])
    # coarse node I sits at fine coordinate 2I
    Z, Y, X = np.meshgrid(*[2.0 * np.arange(n) for n in coarse], indexing="ij")
    c = (a + b[0] * Z + b[1] * Y + b[2] * X)[None]
    Zf, Yf, Xf = np.meshgrid(*[np.arange(n, dtype=float) for n in fine], indexing="ij")
    assert np.allclose(pn.prolong(c, fine)[0], a + b[0] * Zf + b[1] * Yf + b[2] * Xf, atol=1e-12)


def test_restriction_is_scaled_adjoint_and_full_weighting():
    fine, coarse = (9, 7, 5), (5, 4, 3)
    c = _rng().normal(size=(2,) + coarse)
    f = _rng(1).normal(size=(2,) + fine)
    assert float((pn.prolong(c, fine) * f).sum()) == pytest.approx(
        8.0 * float((c * pn.restrict(f, coarse)).sum()), rel=1e-12)
    # full weighting of a constant: weights 1, 1/2, 1/4, 1/8 over 27 fine nodes sum to 8
    r = pn.restrict(np.ones((1,) + fine), coarse)
    assert r[0, 1, 1, 1] == pytest.approx(1.0, abs=1e-14)


def _tiny_net(seed=0, shape=(9, 9, 9), cin=16, cout=4):
    specs = pn.layer_specs(cin, cout)
    w = he_normal_weights([(co, ci) for _, co, ci in specs], seed, last_scale=1.0)
    x = _rng(seed + 1).normal(size=(cin,) + shape)
    return w, x


def test_network_is_positively_homogeneous():
    w, x = _tiny_net()
    y1, _ = pn.forward(w, x, 4)
    y2, _ = pn.forward(w, 3.7 * x, 4)
    assert np.allclose(y2, 3.7 * y1, rtol=1e-12, atol=1e-14)
    assert pn.n_weights(16, 4) == w.size == 6912 * 11 + 3 * 13824 + 1728


@pytest.mark.parametrize("relu_on", [True, False])
def test_gradient_matches_finite_differences_per_layer(relu_on):
    w, x = _tiny_net(shape=(9, 7, 5))
    t = _rng(5).normal(size=(4, 9, 7, 5))
    mask = _rng(6).random(size=(4, 9, 7, 5)) > 0.2

    def loss(wv):
        y, _ = pn.forward(wv, x, 4, relu_on=relu_on)
        return pn.loss_and_grad_y(y, t, mask)[0]

    y, cache = pn.forward(w, x, 4, relu_on=relu_on)
    _, gy = pn.loss_and_grad_y(y, t, mask)
    g = pn.backward(w, cache, gy)
    off = 0
    for name, co, ci in pn.layer_specs(16, 4):
        n = co * ci * 27
        d = np.zeros_like(w)
        d[off:off + n] = _rng(off).normal(size=n)
        # ReLU kinks make any single step unreliable: accept the best of three steps,
        # with the error measured against the layer's gradient scale
        scale = max(abs(float(g @ d)), 1e-3 * float(np.linalg.norm(g[off:off + n]) * np.linalg.norm(d)))
        errs = [abs((loss(w + e * d) - loss(w - e * d)) / (2 * e) - float(g @ d)) / scale
                for e in (1e-5, 1e-6, 1e-7)]
        assert min(errs) <= 1e-6, (name, errs)
        off += n


def test_adam_closed_forms():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = v = np.zeros(3)
    w1, m, v = pn.adam_step(w, g, m, v, 1, 0.01)
    assert np.allclose(w1, w - 0.01 * g / (np.abs(g) + pn.ADAM_EPS), rtol=1e-14)
    # constant gradient: bias-corrected moments stay g and g^2
    wk = w1
    for t in range(2, 6):
        wk, m, v = pn.adam_step(wk, g, m, v, t, 0.01)
    assert np.allclose(wk, w - 5 * 0.01 * g / (np.abs(g) + pn.ADAM_EPS), rtol=1e-12)


def test_pc_pair_round_trip():
    rng = _rng(3)
    shape = (4, 5, 6, 7)
    r, e = rng.normal(size=shape), rng.normal(size=shape)
    dinv = rng.random(size=shape) + 0.5
    dirichlet = rng.random(size=shape) < 0.1
    dinv[dirichlet] = 1.0
    dbar, kc = np.array([1.0, 2.0, 0.5, 3.0]), np.array([0.7, 1.3, 2.0, 0.9])
    rnorm = float(np.linalg.norm(r))
    t = pn.pair_target(r, e, dinv, dirichlet, dbar, rnorm)
    y = t / kc[:, None, None, None]
    z = pn.pc_output(r, dinv, dirichlet, y, dbar, kc, rnorm)
    assert np.allclose(z[~dirichlet], e[~dirichlet], rtol=1e-13, atol=1e-13)
    assert np.array_equal(z[dirichlet], r[dirichlet])
    x = pn.pc_input(r, dinv, [np.ones(shape[1:])], dirichlet, dbar, rnorm)
    assert x.shape[0] == 16 and np.all(x[4] == 1.0) and np.all(x[5:] == 0.0)
    s = np.where(dirichlet, 0.0, dinv * r) / dbar[:, None, None, None]
    assert np.sqrt(np.mean((x[:4] * rnorm / np.sqrt(r.size) - s) ** 2)) < 1e-14


def _spd_like(n, seed):
    rng = _rng(seed)
    A = rng.normal(size=(n, n)) / np.sqrt(n) + 4.0 * np.eye(n)
    return A


def test_fgmres_reduces_to_gmres_with_a_fixed_diagonal():
    A = _spd_like(60, 0)
    b = _rng(1).normal(size=60)
    minv = 1.0 / np.abs(np.diag(A))
    x1, it1, _ = og.gmres(lambda v: A @ v, b, minv, m=10, rtol=1e-10, max_iter=200)
    x2, it2, _ = og.fgmres(lambda v: A @ v, b, lambda v: minv * v, m=10, rtol=1e-10, max_iter=200)
    assert it1 == it2 and np.allclose(x1, x2, rtol=1e-11, atol=1e-12)


def test_fgmres_exact_inverse_and_varying_preconditioner():
    A = _spd_like(40, 2)
    b = _rng(3).normal(size=40)
    Ainv = np.linalg.inv(A)
    x, it, rel = og.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, m=5, rtol=1e-10)
    assert it == 1 and rel <= 1e-10 and np.allclose(x, np.linalg.solve(A, b), rtol=1e-9)
    rng = _rng(4)
    x, it, rel = og.fgmres(lambda v: A @ v, b, lambda v: (0.5 + rng.random(40)) * v, m=8,
                           rtol=1e-10, max_iter=400)
    assert rel <= 1e-10 and np.allclose(x, np.linalg.solve(A, b), rtol=1e-8)


def test_linear_network_and_modulated_input_are_linear_in_r():
    w, _ = _tiny_net(shape=(5, 5, 5))
    rng = _rng(21)
    shape = (4, 5, 5, 5)
    r1, r2 = rng.normal(size=shape), rng.normal(size=shape)
    dinv = rng.random(size=shape) + 0.5
    dirichlet = np.zeros(shape, dtype=bool)
    phases = [np.tanh(rng.normal(size=shape[1:]))]
    dbar, kc = np.ones(4), np.ones(4)

    def M(r):
        return pn.pc_apply(w, r, dinv, phases, dirichlet, dbar, kc, relu_on=False, modulate=True)

    assert np.allclose(M(r1 - 2.5 * r2), M(r1) - 2.5 * M(r2), rtol=1e-10, atol=1e-12)
    x = pn.pc_input(r1, dinv, phases, dirichlet, dbar, 1.0, modulate=True)
    assert np.allclose(x[4:8], x[:4] * 0.5 * (1 + phases[0]), rtol=1e-14) and np.all(x[8:] == 0)


def test_output_smoothing_removes_the_highest_frequency_and_keeps_linear_fields():
    shape = (1, 9, 7, 5)
    zz, yy, xx = np.meshgrid(*[np.arange(k, dtype=float) for k in shape[1:]], indexing="ij")
    r = np.zeros(shape)
    dinv = np.zeros(shape)
    dirichlet = np.zeros(shape, dtype=bool)
    one = np.ones(1)
    lin = (0.3 + zz - 2 * yy + 0.5 * xx)[None]
    # a linear field survives P R wherever the interpolation uses interior coarse
    # nodes only (full weighting is unnormalised at the boundary); the checkerboard
    # is removed there
    z = pn.pc_output(r + 1.0, dinv, dirichlet, lin, one, one, np.sqrt(r.size), smooth=True)
    assert np.allclose(z[0, 2:-2, 2:-2, 2:-2], lin[0, 2:-2, 2:-2, 2:-2], atol=1e-12)
    checker = ((-1.0) ** (zz + yy + xx))[None]
    z = pn.pc_output(r + 1.0, dinv, dirichlet, checker, one, one, np.sqrt(r.size), smooth=True)
    assert np.abs(z[0, 2:-2, 2:-2, 2:-2]).max() < 1e-12
