"""MAC grid and the time-dependent Stokes part of K_E (Sec. 2; Eq. intro_saddle).

Unknowns on the periodic N x N MAC grid, h = L / N:
  u_{i,j} at (i h, (j + 1/2) h), v_{i,j} at ((i + 1/2) h, j h), p_{i,j} at the cell centre.
Global numbering: component c in {0: u, 1: v, 2: p}, index c N^2 + j N + i, all indices mod N.
Operators (centred second order, Sec. 2):
  (D u)_{ij}   = (u_{i+1,j} - u_{ij} + v_{i,j+1} - v_{ij}) / h
  (G p)^u_{ij} = (p_{ij} - p_{i-1,j}) / h,   (G p)^v_{ij} = (p_{ij} - p_{i,j-1}) / h
  (L u)_{ij}   = (u_{i+1,j} + u_{i-1,j} + u_{i,j+1} + u_{i,j-1} - 4 u_{ij}) / h^2  (each component)
  A0 = (rho / dt) I - mu L,   K_E = [[A0 - dt E_E, G], [-D, 0]].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

U, V, P = 0, 1, 2


def idx(N: int, c: int, i, j):
    """Global index of component c at (i, j), periodic."""
    return c * N * N + (np.asarray(j) % N) * N + (np.asarray(i) % N)


def _cells(N):
    j, i = np.divmod(np.arange(N * N), N)
    return i, j


def divergence(N: int, h: float) -> sp.csr_matrix:
    """D: velocity (2N^2) -> cell centres (N^2)."""
    i, j = _cells(N)
    row = np.arange(N * N)
    rows = np.concatenate([row, row, row, row])
    cols = np.concatenate([idx(N, U, i + 1, j), idx(N, U, i, j), idx(N, V, i, j + 1), idx(N, V, i, j)])
    vals = np.concatenate([np.full(N * N, 1.0 / h), np.full(N * N, -1.0 / h),
                           np.full(N * N, 1.0 / h), np.full(N * N, -1.0 / h)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(N * N, 2 * N * N))


def gradient(N: int, h: float) -> sp.csr_matrix:
    """G: cell centres (N^2) -> velocity faces (2N^2); indices local to the pressure block."""
    i, j = _cells(N)
    ru = idx(N, U, i, j)
    rv = idx(N, V, i, j)
    rows = np.concatenate([ru, ru, rv, rv])
    cols = np.concatenate([j * N + i, j * N + (i - 1) % N, j * N + i, ((j - 1) % N) * N + i])
    vals = np.concatenate([np.full(N * N, 1.0 / h), np.full(N * N, -1.0 / h),
                           np.full(N * N, 1.0 / h), np.full(N * N, -1.0 / h)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * N * N, N * N))


def laplacian(N: int, h: float) -> sp.csr_matrix:
    """Vector 5-point Laplacian on both velocity components."""
    i, j = _cells(N)
    rows, cols, vals = [], [], []
    for c in (U, V):
        r = idx(N, c, i, j)
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            rows.append(r)
            cols.append(idx(N, c, i + di, j + dj))
            vals.append(np.full(N * N, 1.0 / h ** 2))
        rows.append(r)
        cols.append(r)
        vals.append(np.full(N * N, -4.0 / h ** 2))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(2 * N * N, 2 * N * N))


def A0(N: int, h: float, rho: float, dt: float, mu: float) -> sp.csr_matrix:
    """Time-discrete momentum matrix A0 = (rho/dt) I - mu L (Eq. intro_saddle)."""
    return (rho / dt) * sp.identity(2 * N * N, format="csr") - mu * laplacian(N, h)


def reduced_operator(N: int, h: float, rho: float, dt: float, mu: float,
                     EE: sp.spmatrix | None) -> sp.csr_matrix:
    """K_E = [[A0 - dt E_E, G], [-D, 0]] on U_h x P_h coefficient space (Eq. Eul_schur)."""
    A = A0(N, h, rho, dt, mu)
    if EE is not None:
        A = A - dt * EE
    G = gradient(N, h)
    D = divergence(N, h)
    return sp.bmat([[A, G], [-D, None]], format="csr")
