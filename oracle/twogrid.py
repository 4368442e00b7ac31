"""Two-grid iteration matrix and its spectrum (Sec. 5.1, Table 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With two levels (the fine grid and the coarsest, solved directly) the V-cycle is the two-grid
preconditioner B^TG, and the stationary two-grid iteration has the error propagation
T = I - B^TG K_E.  The paper reports rho(T) and the smallest and largest |lambda(B^TG K_E)|.

On the periodic grid K_E annihilates the constant pressure and B^TG returns mean-zero
pressure, so B^TG K_E maps everything into the mean-zero subspace and is zero on the
constant: its spectrum is {0} together with the spectrum of its restriction to U_h x P_h
(Sec. 2's restriction, the reading taken here).  Both are computed with dense matrices:
column i of B^TG K_E is B^TG applied to K_E e_i.
"""
from __future__ import annotations

import numpy as np


def mean_zero_basis(N: int) -> np.ndarray:
    """Orthonormal basis (columns) of the vectors whose pressure block has zero mean."""
    n = 3 * N * N
    c = np.zeros(n)
    c[2 * N * N:] = 1.0 / N
    # Householder reflector mapping c to e_0; its remaining columns span the complement of c
    v = c.copy()
    v[0] -= 1.0
    H = np.eye(n) - 2.0 * np.outer(v, v) / (v @ v)
    return H[:, 1:]


def preconditioned_operator(apply_K, apply_B, n: int) -> np.ndarray:
    """Dense B K, column by column."""
    BK = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[i] = 1.0
        BK[:, i] = apply_B(apply_K(e))
        e[i] = 0.0
    return BK


def spectrum_summary(BK: np.ndarray, N: int) -> dict:
    """rho(T) and min / max |lambda(B K)| on the mean-zero subspace."""
    Q = mean_zero_basis(N)
    lam = np.linalg.eigvals(Q.T @ BK @ Q)
    return {"rho_T": float(np.max(np.abs(1.0 - lam))),
            "min_abs_lambda": float(np.min(np.abs(lam))),
            "max_abs_lambda": float(np.max(np.abs(lam)))}
