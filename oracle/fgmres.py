"""Right-preconditioned flexible GMRES (Sec. 5): zero initial guess unless given, Euclidean
norms, no restarts, stop when ||r_k||_2 <= rtol * ||ref||_2.

Readings: modified Gram-Schmidt Arnoldi and Givens rotations (the paper names neither);
the stopping reference is ||b|| by default (equal to ||r_0|| for the paper's zero guess),
and ||r_0|| on request.
"""
from __future__ import annotations

import math

import numpy as np


def fgmres(apply_K, b, precond, x0=None, rtol=1e-10, maxit=60, ref="b"):
    """Returns (x, info) with info = {iters, converged, relres_est, relres_true, history}."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_K(x)
    beta = float(np.linalg.norm(r))
    ref_norm = float(np.linalg.norm(b)) if ref == "b" else beta
    hist = [beta / ref_norm if ref_norm > 0 else 0.0]
    if ref_norm == 0.0 or beta <= rtol * ref_norm:
        return x, {"iters": 0, "converged": True, "relres_est": hist[0],
                   "relres_true": hist[0], "history": hist}
    n = b.shape[0]
    Vb = np.zeros((maxit + 1, n))
    Zb = np.zeros((maxit, n))
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    Vb[0] = r / beta
    k_done = 0
    converged = False
    for k in range(maxit):
        Zb[k] = precond(Vb[k])
        w = apply_K(Zb[k])
        for i in range(k + 1):
            H[i, k] = float(np.dot(w, Vb[i]))
            w = w - H[i, k] * Vb[i]
        H[k + 1, k] = float(np.linalg.norm(w))
        if H[k + 1, k] != 0.0:
            Vb[k + 1] = w / H[k + 1, k]
        for i in range(k):
            t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
            H[i, k] = t
        d = math.hypot(H[k, k], H[k + 1, k])
        cs[k] = H[k, k] / d
        sn[k] = H[k + 1, k] / d
        H[k, k] = d
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        k_done = k + 1
        hist.append(abs(g[k + 1]) / ref_norm)
        if abs(g[k + 1]) <= rtol * ref_norm:
            converged = True
            break
    y = np.zeros(k_done)
    for i in range(k_done - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:k_done] @ y[i + 1:]) / H[i, i]
    x = x + Zb[:k_done].T @ y
    true = float(np.linalg.norm(b - apply_K(x))) / ref_norm
    return x, {"iters": k_done, "converged": converged, "relres_est": hist[-1],
               "relres_true": true, "history": hist}
