"""Learned right preconditioner for the NS block: a 3D convolutional U-Net (oracle).

Test infrastructure only (see oracle/__init__.py).

The paper solves each block with GMRES (Section 2.5, second remark) and prescribes no
preconditioner.  This module defines, in plain float64 numpy, the small network that
the GPU library trains and applies as a flexible right preconditioner inside FGMRES
(Saad's flexible GMRES, `oracle.gmres.fgmres`), together with everything around it:

  * the grids: level 0 is the mesh's node grid; level l+1 keeps every other node of
    level l, so a level with n nodes along an axis has n // 2 + 1 coarse nodes
    (65 -> 33 -> 17 -> 9 for a 64-element axis);
  * P (prolongation) is Q1 interpolation from a coarse node grid to the fine one
    (injection at even fine nodes, the average of the two neighbours at odd ones,
    tensor product in 3D); R (restriction) is (1/8) P^T;
  * conv: 3x3x3 cross-correlation with zero padding, no bias, weights W[co, ci, kz, ky, kx];
  * the network, 4 levels, 16 channels:
        a_l = relu(conv(x_l)), e_l = relu(conv(a_l)), x_{l+1} = R e_l      (l = 0, 1, 2)
        a_3 = relu(conv(x_3)), d_3 = relu(conv(a_3))
        b_l = relu(conv(cat(e_l, P d_{l+1}))), d_l = relu(conv(b_l))       (l = 2, 1, 0)
        y   = conv(d_0)
    15 convolutions, without biases, so the network is positively homogeneous in x;
  * the loss: mean squared error over the non-Dirichlet nodes and the block's
    components, and its gradient with respect to every weight (reverse mode written
    out layer by layer);
  * Adam (Kingma & Ba 2015) with bias correction;
  * the preconditioner apply: the input channels are the Jacobi-scaled residual
    normalised to unit RMS plus the phase indicators, the output is added to the
    Jacobi step (z = D^{-1} r + correction), Dirichlet rows pass r through;
  * training pairs: for checkpoints x_k of a converged solve of A x = b with final
    iterate x*, the pair (r_k - r*, x* - x_k) satisfies A (x* - x_k) = r_k - r* exactly.

`quant="bf16"` rounds, at the same places as the GPU kernels store them, the weights,
the activations, the restriction/prolongation results and the back-propagated
activation gradients to bfloat16 (round to nearest even); all arithmetic between those
points stays float64.  `quant="bf16-f32"` rounds at the same places but accumulates
the convolutions in float32: the spread between the two measures how far two correct
implementations of the bfloat16 network can drift apart through rounding alone (the
tests take their tolerances from it).  `quant=None` is the float64 network.

Parity pins: tests/test_oracle_pcnet.py (brute-force convolution, adjoint identities,
Q1 reproduction of linear fields, finite-difference gradients, Adam closed forms).
"""
from __future__ import annotations

import numpy as np

LEVELS = 4
CH = 16
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


# --------------------------------------------------------------------- rounding
def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via float32; returns float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def _q(a, quant):
    return bf16(a) if quant in ("bf16", "bf16-f32") else a


def _acc(quant):
    return np.float32 if quant == "bf16-f32" else np.float64


# ------------------------------------------------------------------------ grids
def level_shapes(shape0) -> list:
    """Node-grid shapes (nz, ny, nx) of the 4 levels."""
    out = [tuple(shape0)]
    for _ in range(LEVELS - 1):
        out.append(tuple(n // 2 + 1 for n in out[-1]))
    return out


def p1d(nf: int, nc: int) -> np.ndarray:
    """1D Q1 interpolation matrix from nc coarse nodes (spacing 2) to nf fine nodes."""
    P = np.zeros((nf, nc))
    for i in range(nf):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, (i - 1) // 2] = 0.5
            P[i, (i + 1) // 2] = 0.5
    return P


def prolong(c: np.ndarray, fine_shape) -> np.ndarray:
    """P c for c[C, nz, ny, nx] on the coarse grid."""
    Pz, Py, Px = (p1d(nf, nc) for nf, nc in zip(fine_shape, c.shape[1:]))
    return np.einsum("zc,yb,xa,kcba->kzyx", Pz, Py, Px, c)


def restrict(f: np.ndarray, coarse_shape) -> np.ndarray:
    """R f = (1/8) P^T f."""
    Pz, Py, Px = (p1d(nf, nc) for nf, nc in zip(f.shape[1:], coarse_shape))
    return np.einsum("zc,yb,xa,kzyx->kcba", Pz, Py, Px, f) / 8.0


# ----------------------------------------------------------------- convolutions
def conv3(x: np.ndarray, W: np.ndarray, acc=np.float64) -> np.ndarray:
    """y[o, v] = sum_{i, k} W[o, i, k] x[i, v + k - 1], zero outside the grid
    (accumulated in the floating type `acc`, returned as float64)."""
    _, nz, ny, nx = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1))).astype(acc)
    W = W.astype(acc)
    y = np.zeros((W.shape[0], nz, ny, nx), dtype=acc)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                y += np.einsum("oi,izyx->ozyx", W[:, :, kz, ky, kx],
                               xp[:, kz:kz + nz, ky:ky + ny, kx:kx + nx])
    return y.astype(np.float64)


def conv3_adjoint(g: np.ndarray, W: np.ndarray, acc=np.float64) -> np.ndarray:
    """The adjoint of x -> conv3(x, W) applied to g[o, v]."""
    _, nz, ny, nx = g.shape
    g, W = g.astype(acc), W.astype(acc)
    xp = np.zeros((W.shape[1], nz + 2, ny + 2, nx + 2), dtype=acc)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                xp[:, kz:kz + nz, ky:ky + ny, kx:kx + nx] += np.einsum(
                    "oi,ozyx->izyx", W[:, :, kz, ky, kx], g)
    return xp[:, 1:-1, 1:-1, 1:-1].astype(np.float64)


def conv3_wgrad(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """dW[o, i, k] = sum_v g[o, v] x[i, v + k - 1] (the gradient of <g, conv3(x, W)>)."""
    _, nz, ny, nx = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dW = np.zeros((g.shape[0], x.shape[0], 3, 3, 3))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                dW[:, :, kz, ky, kx] = np.einsum("ozyx,izyx->oi", g,
                                                 xp[:, kz:kz + nz, ky:ky + ny, kx:kx + nx])
    return dW


# ---------------------------------------------------------------------- network
def layer_specs(cin0: int, cout: int) -> list:
    """(name, out channels, in channels) of the 15 convolutions, in storage order."""
    s = [("enc0a", CH, cin0), ("enc0b", CH, CH)]
    for lv in (1, 2):
        s += [(f"enc{lv}a", CH, CH), (f"enc{lv}b", CH, CH)]
    s += [("bota", CH, CH), ("botb", CH, CH)]
    for lv in (2, 1, 0):
        s += [(f"dec{lv}a", CH, 2 * CH), (f"dec{lv}b", CH, CH)]
    s += [("out", cout, CH)]
    return s


def n_weights(cin0: int, cout: int) -> int:
    return sum(co * ci * 27 for _, co, ci in layer_specs(cin0, cout))


def unflatten(w: np.ndarray, cin0: int, cout: int) -> dict:
    """Flat weight vector -> {name: W[co, ci, 3, 3, 3]} (row-major in that order)."""
    out, off = {}, 0
    for name, co, ci in layer_specs(cin0, cout):
        n = co * ci * 27
        out[name] = np.asarray(w[off:off + n], dtype=np.float64).reshape(co, ci, 3, 3, 3)
        off += n
    assert off == w.size
    return out


def flatten(Ws: dict, cin0: int, cout: int) -> np.ndarray:
    return np.concatenate([Ws[name].ravel() for name, _, _ in layer_specs(cin0, cout)])


def forward(w: np.ndarray, x0: np.ndarray, cout: int, quant=None, relu_on: bool = True):
    """y = network(x0); x0[cin0, nz, ny, nx].  Returns (y, cache).  relu_on=False
    drops every ReLU: the network is then a linear operator of x0 (a learned
    multigrid-like cycle of convolutions, restrictions and prolongations)."""
    cin0 = x0.shape[0]
    W = {k: _q(v, quant) for k, v in unflatten(w, cin0, cout).items()}
    shapes = level_shapes(x0.shape[1:])
    relu = (lambda a: np.maximum(a, 0.0)) if relu_on else (lambda a: a)  # noqa: E731
    conv = lambda a, Wl: conv3(a, Wl, _acc(quant))  # noqa: E731
    c = {"x0": _q(x0, quant)}
    for lv in range(3):
        c[f"a{lv}"] = _q(relu(conv(c[f"x{lv}"], W[f"enc{lv}a"])), quant)
        c[f"e{lv}"] = _q(relu(conv(c[f"a{lv}"], W[f"enc{lv}b"])), quant)
        c[f"x{lv + 1}"] = _q(restrict(c[f"e{lv}"], shapes[lv + 1]), quant)
    c["a3"] = _q(relu(conv(c["x3"], W["bota"])), quant)
    c["d3"] = _q(relu(conv(c["a3"], W["botb"])), quant)
    for lv in (2, 1, 0):
        up = _q(prolong(c[f"d{lv + 1}"], shapes[lv]), quant)
        c[f"c{lv}"] = np.concatenate([c[f"e{lv}"], up])
        c[f"b{lv}"] = _q(relu(conv(c[f"c{lv}"], W[f"dec{lv}a"])), quant)
        c[f"d{lv}"] = _q(relu(conv(c[f"b{lv}"], W[f"dec{lv}b"])), quant)
    y = conv(c["d0"], W["out"])
    c["W"] = W
    c["relu_on"] = relu_on
    return y, c


def loss_and_grad_y(y: np.ndarray, t: np.ndarray, mask: np.ndarray):
    """L = sum over the rows where mask[c, v] is set of (y - t)^2, divided by the
    number of those rows, and dL/dy (mask: the non-Dirichlet rows)."""
    cnt = float(mask.sum())
    d = (y - t) * mask
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def backward(w: np.ndarray, cache: dict, gy: np.ndarray, quant=None) -> np.ndarray:
    """dL/dw (flat, storage order) from dL/dy, by reverse mode through `forward`."""
    W = cache["W"]
    cin0 = cache["x0"].shape[0]
    cout = gy.shape[0]
    shapes = level_shapes(cache["x0"].shape[1:])
    gW = {}
    if cache["relu_on"]:
        mask = lambda g, a: g * (a > 0)  # noqa: E731  (relu' from the stored output)
    else:
        mask = lambda g, a: g  # noqa: E731
    conv3_adj = lambda g, Wl: conv3_adjoint(g, Wl, _acc(quant))  # noqa: E731
    g = _q(gy, quant)
    gW["out"] = conv3_wgrad(cache["d0"], g)
    g_d = _q(mask(conv3_adj(g, W["out"]), cache["d0"]), quant)
    g_e = {}
    for lv in (0, 1, 2):
        gW[f"dec{lv}b"] = conv3_wgrad(cache[f"b{lv}"], g_d)
        g_b = _q(mask(conv3_adj(g_d, W[f"dec{lv}b"]), cache[f"b{lv}"]), quant)
        gW[f"dec{lv}a"] = conv3_wgrad(cache[f"c{lv}"], g_b)
        g_c = _q(conv3_adj(g_b, W[f"dec{lv}a"]), quant)
        g_e[lv] = g_c[:CH]
        # adjoint of P is 8 R
        g_d = _q(mask(8.0 * restrict(g_c[CH:], shapes[lv + 1]), cache[f"d{lv + 1}"]), quant)
    gW["botb"] = conv3_wgrad(cache["a3"], g_d)
    g_a = _q(mask(conv3_adj(g_d, W["botb"]), cache["a3"]), quant)
    gW["bota"] = conv3_wgrad(cache["x3"], g_a)
    g_x = _q(conv3_adj(g_a, W["bota"]), quant)
    for lv in (2, 1, 0):
        # adjoint of R is (1/8) P; e_l also feeds the decoder's concatenation
        g_el = _q(mask(g_e[lv] + prolong(g_x, shapes[lv]) / 8.0, cache[f"e{lv}"]), quant)
        gW[f"enc{lv}b"] = conv3_wgrad(cache[f"a{lv}"], g_el)
        g_a = _q(mask(conv3_adj(g_el, W[f"enc{lv}b"]), cache[f"a{lv}"]), quant)
        gW[f"enc{lv}a"] = conv3_wgrad(cache[f"x{lv}"], g_a)
        if lv > 0:
            g_x = _q(conv3_adj(g_a, W[f"enc{lv}a"]), quant)
    return flatten(gW, cin0, cout)


# ------------------------------------------------------------------------- Adam
def adam_step(w, g, m, v, t: int, lr: float):
    """One Adam update at step t >= 1; returns (w, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mh = m / (1.0 - ADAM_B1 ** t)
    vh = v / (1.0 - ADAM_B2 ** t)
    return w - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


# ------------------------------------------------------- preconditioner apply
def pc_input(r, dinv, phases, dirichlet, dbar, rnorm, quant=None, modulate=False):
    """Network input channels [16 k, nz, ny, nx] from a block residual r[ncomp][...]:
    s_c = (D^{-1} r)_c * sqrt(n_rows) / (rnorm * dbar_c) on non-Dirichlet rows (0 on
    Dirichlet rows), followed by either the indicators `phases` themselves or, with
    modulate=True, the products s_c * (1 + phi) / 2 for every indicator in `phases`
    (the input, and a network without ReLU, then stay linear in r); zero padded."""
    ncomp = r.shape[0]
    g = np.sqrt(r.size) / rnorm
    s = np.where(dirichlet, 0.0, dinv * r)
    chans = [s[c] * g / dbar[c] for c in range(ncomp)]
    if modulate:
        chans += [chans[c] * 0.5 * (1.0 + ph) for ph in phases for c in range(ncomp)]
    else:
        chans += list(phases)
    cin = -(-len(chans) // CH) * CH
    x = np.zeros((cin,) + r.shape[1:])
    x[:len(chans)] = chans
    return _q(x, quant)


def pc_output(r, dinv, dirichlet, y, dbar, kc, rnorm, smooth=False):
    """z = D^{-1} r + (rnorm / sqrt(n_rows)) dbar_c kc_c y_c; z = r on Dirichlet rows.
    smooth=True first replaces y by P R y (full weighting to the next coarser node grid
    and Q1 interpolation back): that removes the high-frequency part of the network's
    output, where its bfloat16 rounding noise lives and where the operator's large
    eigenvalues would amplify it."""
    ncomp = r.shape[0]
    if smooth:
        coarse = tuple(k // 2 + 1 for k in y.shape[1:])
        y = prolong(restrict(y, coarse), y.shape[1:])
    h = rnorm / np.sqrt(r.size)
    z = dinv * r + np.stack([h * dbar[c] * kc[c] * y[c] for c in range(ncomp)])
    return np.where(dirichlet, r, z)


def pc_apply(w, r, dinv, phases, dirichlet, dbar, kc, quant=None, relu_on=True, modulate=False, smooth=False):
    rnorm = float(np.linalg.norm(r))
    if rnorm == 0.0:
        return np.zeros_like(r)
    x = pc_input(r, dinv, phases, dirichlet, dbar, rnorm, quant, modulate)
    y, _ = forward(w, x, r.shape[0], quant, relu_on)
    return pc_output(r, dinv, dirichlet, y, dbar, kc, rnorm, smooth)


def pair_target(r, e, dinv, dirichlet, dbar, rnorm):
    """Training target t_c = (e - D^{-1} r)_c sqrt(n_rows) / (rnorm dbar_c) (0 on
    Dirichlet rows): pc_output with y_c = t_c / kc_c returns e on non-Dirichlet rows."""
    ncomp = r.shape[0]
    g = np.sqrt(r.size) / rnorm
    t = np.stack([(e[c] - dinv[c] * r[c]) * g / dbar[c] for c in range(ncomp)])
    return np.where(dirichlet, 0.0, t)
