"""Restarted GMRES with right preconditioning and modified Gram-Schmidt (oracle).

Test infrastructure only (see oracle/__init__.py).

The paper solves every block's linear system with GMRES (Section 2.5, second remark).
Textbook restarted GMRES(m) (Saad & Schultz): x_0 = 0, Arnoldi with modified
Gram-Schmidt on A M^{-1}, Givens rotations on the Hessenberg matrix, restart every m
iterations, stop when ||b - A x|| / ||b|| <= rtol (the rotated residual estimate is
used inside a cycle; the true residual is recomputed at each restart).
"""
from __future__ import annotations

import numpy as np


def gmres(apply_A, b: np.ndarray, minv=None, m: int = 30, rtol: float = 1e-8,
          max_iter: int = 1000):
    """Returns (x, iterations, final relative residual)."""
    n = b.shape[0]
    minv = np.ones(n) if minv is None else minv
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b.copy()
    rel = 1.0
    while it < max_iter:
        beta = float(np.linalg.norm(r))
        rel = beta / bnorm
        if rel <= rtol:
            break
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            w = apply_A(minv * V[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_end = j + 1
            if abs(g[j + 1]) / bnorm <= rtol or it >= max_iter or H[j, j] == 0.0:
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_end], y[i + 1:j_end])) / H[i, i]
        x = x + minv * (V[:j_end].T @ y)
        r = b - apply_A(x)
    rel = float(np.linalg.norm(r)) / bnorm
    return x, it, rel


def fgmres(apply_A, b: np.ndarray, apply_M, m: int = 30, rtol: float = 1e-8,
           max_iter: int = 1000):
    """Flexible GMRES(m) (Saad 1993): the right preconditioner M may change from one
    iteration to the next (a trained network is not a fixed linear map), so the
    preconditioned directions z_j = M(v_j) are kept and the update is x += Z y.
    Modified Gram-Schmidt and Givens rotations as in `gmres`.
    Returns (x, iterations, final relative residual)."""
    n = b.shape[0]
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b.copy()
    rel = 1.0
    while it < max_iter:
        beta = float(np.linalg.norm(r))
        rel = beta / bnorm
        if rel <= rtol:
            break
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = apply_M(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_end = j + 1
            if abs(g[j + 1]) / bnorm <= rtol or it >= max_iter or H[j, j] == 0.0:
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_end], y[i + 1:j_end])) / H[i, i]
        x = x + Z[:j_end].T @ y
        r = b - apply_A(x)
    rel = float(np.linalg.norm(r)) / bnorm
    return x, it, rel
