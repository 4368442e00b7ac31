"""Nonlinear fiber force law of the flow-past-a-fiber benchmark (Sec. 5.3) and its Newton tangent.

TEST INFRASTRUCTURE ONLY (see the package docstring).

An open fiber of M markers with links D_k = X_{k+1} - X_k (k = 0 .. M-2) and spacing ds:

  bending     E_b = EI / (2 ds^5)  sum_{k=0}^{M-3} (D_k x D_{k+1})^2,   a x b = a_x b_y - a_y b_x
  stretching  E_s = K_s / (2 ds)   sum_{k=0}^{M-2} (|D_k| - ds)^2
  clamp       E_p = K_p / 2 |X_m - X_c|^2
              E_t = K_t / 2 |(X_{m+1} - X_{m-1}) / (2 ds) - e_x|^2
  force       F = -(1/ds) grad_X (E_b + E_s + E_p + E_t)
  tangent     E = dF/dX = -(1/ds) Hess_X (E_b + E_s + E_p + E_t)   (2M x 2M, symmetric)

The tangent replaces the linear laws' E in the Eulerian system (Eq. intro_saddle) at each
Newton step; unlike them it couples the x and y components.  Vectors are component-major
(index c M + k), as everywhere in the oracle.  m is the midpoint marker (M odd), X_c its
prescribed position and e_x = (1, 0).

Each term's gradient and Hessian is written out from its definition (chain rule on the
link vectors); the pins check them against finite differences of the energy, against the
invariances of E_b and E_s, and, at the straight reference configuration, against the
textbook linearisations (open second and fourth differences).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class FiberParams:
    M: int
    ds: float
    EI: float
    K_s: float
    K_p: float
    K_t: float
    X_c: tuple = (1.0, 1.5)

    @property
    def m(self) -> int:
        return self.M // 2


def _split(X):
    """(M, 2) marker array from a component-major vector or an (M, 2) array."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        M = X.size // 2
        return np.stack([X[:M], X[M:]], 1)
    return X


def _cm(G):
    """Component-major vector from an (M, 2) array."""
    return np.concatenate([G[:, 0], G[:, 1]])


def energy(p: FiberParams, X) -> dict:
    """The four energies of Sec. 5.3."""
    X = _split(X)
    D = X[1:] - X[:-1]
    cr = D[:-1, 0] * D[1:, 1] - D[:-1, 1] * D[1:, 0]
    Eb = p.EI / (2.0 * p.ds ** 5) * float(np.sum(cr * cr))
    L = np.sqrt(np.sum(D * D, 1))
    Es = p.K_s / (2.0 * p.ds) * float(np.sum((L - p.ds) ** 2))
    m = p.m
    dp = X[m] - np.asarray(p.X_c)
    Ep = 0.5 * p.K_p * float(dp @ dp)
    tv = (X[m + 1] - X[m - 1]) / (2.0 * p.ds) - np.array([1.0, 0.0])
    Et = 0.5 * p.K_t * float(tv @ tv)
    return {"bend": Eb, "stretch": Es, "position": Ep, "tangent": Et, "total": Eb + Es + Ep + Et}


# the scalar cross product c = a x b and its derivatives with respect to (a, b) in R^4
_DC_DA = lambda b: np.array([b[1], -b[0]])   # dc/da
_DC_DB = lambda a: np.array([-a[1], a[0]])   # dc/db
# d^2 c / d(a,b)^2: constant, c = a0 b1 - a1 b0
_D2C = np.array([[0, 0, 0, 1],
                 [0, 0, -1, 0],
                 [0, -1, 0, 0],
                 [1, 0, 0, 0]], dtype=np.float64)


def gradient(p: FiberParams, X) -> np.ndarray:
    """grad_X of the total energy, component-major (2M)."""
    X = _split(X)
    M = X.shape[0]
    G = np.zeros((M, 2))
    D = X[1:] - X[:-1]
    # bending: term k depends on D_k = X_{k+1} - X_k and D_{k+1} = X_{k+2} - X_{k+1}
    cb = p.EI / p.ds ** 5
    for k in range(M - 2):
        a, b = D[k], D[k + 1]
        c = a[0] * b[1] - a[1] * b[0]
        ga, gb = cb * c * _DC_DA(b), cb * c * _DC_DB(a)     # d(EI/(2ds^5) c^2)/da, /db
        G[k] -= ga
        G[k + 1] += ga - gb
        G[k + 2] += gb
    # stretching: d/dD (|D| - ds)^2 / 2 = (|D| - ds) D / |D|
    cs = p.K_s / p.ds
    for k in range(M - 1):
        d = D[k]
        L = np.sqrt(d @ d)
        g = cs * (L - p.ds) * d / L
        G[k] -= g
        G[k + 1] += g
    m = p.m
    G[m] += p.K_p * (X[m] - np.asarray(p.X_c))
    tv = (X[m + 1] - X[m - 1]) / (2.0 * p.ds) - np.array([1.0, 0.0])
    gt = p.K_t * tv / (2.0 * p.ds)
    G[m + 1] += gt
    G[m - 1] -= gt
    return _cm(G)


def hessian(p: FiberParams, X) -> sp.csr_matrix:
    """Hess_X of the total energy (2M x 2M, component-major, symmetric)."""
    X = _split(X)
    M = X.shape[0]
    H = np.zeros((M, 2, M, 2))
    D = X[1:] - X[:-1]

    def add_link_pair(k, Hab):
        """Add a 4x4 Hessian in (D_k, D_{k+1}) to the markers k, k+1, k+2 (D_k = X_{k+1} - X_k)."""
        # dD_k/dX: -I at k, +I at k+1; dD_{k+1}/dX: -I at k+1, +I at k+2
        S = {0: [(k, -1.0), (k + 1, 1.0)], 1: [(k + 1, -1.0), (k + 2, 1.0)]}
        for ia in (0, 1):
            for ib in (0, 1):
                blk = Hab[2 * ia:2 * ia + 2, 2 * ib:2 * ib + 2]
                for (ma, sa) in S[ia]:
                    for (mb, sb) in S[ib]:
                        H[ma, :, mb, :] += sa * sb * blk

    cb = p.EI / p.ds ** 5
    for k in range(M - 2):
        a, b = D[k], D[k + 1]
        c = a[0] * b[1] - a[1] * b[0]
        dc = np.concatenate([_DC_DA(b), _DC_DB(a)])
        # d^2 (c^2 / 2) = dc dc^T + c d^2 c
        add_link_pair(k, cb * (np.outer(dc, dc) + c * _D2C))
    cs = p.K_s / p.ds
    for k in range(M - 1):
        d = D[k]
        L = np.sqrt(d @ d)
        u = d / L
        # d^2/dD^2 (|D| - ds)^2 / 2 = u u^T + (|D| - ds)/|D| (I - u u^T)
        Hd = cs * (np.outer(u, u) + (L - p.ds) / L * (np.eye(2) - np.outer(u, u)))
        for (ma, sa) in ((k, -1.0), (k + 1, 1.0)):
            for (mb, sb) in ((k, -1.0), (k + 1, 1.0)):
                H[ma, :, mb, :] += sa * sb * Hd
    m = p.m
    H[m, :, m, :] += p.K_p * np.eye(2)
    ct = p.K_t / (2.0 * p.ds) ** 2
    for (ma, sa) in ((m + 1, 1.0), (m - 1, -1.0)):
        for (mb, sb) in ((m + 1, 1.0), (m - 1, -1.0)):
            H[ma, :, mb, :] += sa * sb * ct * np.eye(2)
    # (marker, component) -> component-major
    Hc = H.transpose(1, 0, 3, 2).reshape(2 * M, 2 * M)
    return sp.csr_matrix(Hc)


def force(p: FiberParams, X) -> np.ndarray:
    """F = -(1/ds) grad_X E (Sec. 5.3), component-major."""
    return -gradient(p, X) / p.ds


def tangent(p: FiberParams, X) -> sp.csr_matrix:
    """E = dF/dX = -(1/ds) Hess_X E: the Newton tangent that takes E's place in K_E."""
    return (-hessian(p, X) / p.ds).tocsr()


def tangent_pattern(p: FiberParams) -> sp.csr_matrix:
    """Structural pattern of the tangent at any configuration: bending term k couples the
    markers k, k+1, k+2 (so every pair within two links; the clamp's m -+ 1 pair is one of
    them), stretching the ends of a link; x and y are coupled throughout."""
    M = p.M
    w = 2 if M >= 3 else 1
    k = np.arange(M)
    B = np.abs(k[:, None] - k[None, :]) <= w
    return sp.csr_matrix(np.kron(np.ones((2, 2), dtype=bool), B))


def straight_fiber(M: int, ds: float, centre=(1.0, 1.5)) -> np.ndarray:
    """The straight horizontal reference configuration of Sec. 5.3, centred on the midpoint."""
    x = centre[0] + (np.arange(M) - M // 2) * ds
    return np.stack([x, np.full(M, centre[1])], 1)


def paper_params(N: int) -> FiberParams:
    """Sec. 5.3's parameters at h = 1/N (domain (0,2)^2 with 2N x 2N cells): ds = h/2,
    EI = 2.63672e-2; K_s, K_p, K_t = 375, 1200, 7.03125 at N = 64 and doubled whenever h is
    halved (proportional to N); M markers spanning the length 0.375 (13, 25, 49, 97 markers
    at N = 16, 32, 64, 128)."""
    h = 1.0 / N
    ds = h / 2.0
    M = int(round(0.375 / ds)) + 1
    f = N / 64.0
    return FiberParams(M=M, ds=ds, EI=2.63672e-2, K_s=375.0 * f, K_p=1200.0 * f, K_t=7.03125 * f)
