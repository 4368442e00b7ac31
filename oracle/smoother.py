"""Patch relaxation of Sec. 3.3 and the weighted additive form of Eq. (additive_cav_saddle).

Local factorisation (Sec. 3.3): K_{E,p} = R_p K_E R_p^T; one pass of max-norm row and
column equilibration, then LU.  Readings where the paper is silent:
  * row scales first, s_r[i] = 1 / max_j |K_ij|, then column scales of diag(s_r) K,
    s_c[j] = 1 / max_i |s_r[i] K_ij|; each scale rounded to the power of two 2^-e where
    max = m 2^e, m in [1/2, 1) -- so the scaling itself is exact in FP64;
  * LU with partial pivoting, the first row of maximal modulus taking ties;
  * the stored inverse X_p = (diag(s_r) K_{E,p} diag(s_c))^-1 is obtained by solving
    LU X = P I (forward, then back substitution);  delta_p = diag(s_c) X_p diag(s_r) r_p;
  * a patch that holds every pressure unknown of a periodic level has K_{E,p} singular on
    constant pressure; it is solved with the bordered matrix [[K_p, e], [e^T, 0]], e the
    indicator of its pressure slots (the restriction to U_h x P_h of Sec. 2).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


class SingularPatch(ArithmeticError):
    pass


def local_matrix(KE: sp.csr_matrix, dofs: np.ndarray) -> np.ndarray:
    """K_{E,p} = R_p K_E R_p^T as a dense array."""
    return KE[dofs][:, dofs].toarray()


def _pow2_recip(m: float) -> float:
    if m == 0.0:
        raise SingularPatch("zero row or column")
    _, e = math.frexp(m)
    return math.ldexp(1.0, -e)


def equilibrate(K: np.ndarray):
    """One pass of max-norm row then column equilibration; returns (s_r, s_c)."""
    s_r = np.array([_pow2_recip(float(np.max(np.abs(K[i, :])))) for i in range(K.shape[0])])
    K1 = s_r[:, None] * K
    s_c = np.array([_pow2_recip(float(np.max(np.abs(K1[:, j])))) for j in range(K.shape[1])])
    return s_r, s_c


def lu_factor(A: np.ndarray):
    """Gaussian elimination with partial pivoting: P A = L U packed into one array."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0.0:
            raise SingularPatch(f"zero pivot at column {k}")
        if p != k:
            A[[k, p]] = A[[p, k]]
            perm[[k, p]] = perm[[p, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, perm


def lu_inverse(LU: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """Solve L U X = P I column block by column block."""
    n = LU.shape[0]
    Y = np.eye(n)[perm]
    for i in range(n):
        Y[i] -= LU[i, :i] @ Y[:i]
    for i in range(n - 1, -1, -1):
        Y[i] = (Y[i] - LU[i, i + 1:] @ Y[i + 1:]) / LU[i, i]
    return Y


class PatchSolver:
    """Stored local solve of one patch: delta = s_c * (X (s_r * r_p))."""

    def __init__(self, KE: sp.csr_matrix, dofs: np.ndarray, n_total_pressure: int | None = None,
                 pressure_start: int | None = None):
        self.dofs = np.asarray(dofs, dtype=np.int64)
        K = local_matrix(KE, self.dofs)
        self.bordered = False
        if n_total_pressure is not None:
            npres = int(np.sum(self.dofs >= pressure_start))
            if npres == n_total_pressure:
                e = (self.dofs >= pressure_start).astype(np.float64)
                n = K.shape[0]
                Kb = np.zeros((n + 1, n + 1))
                Kb[:n, :n] = K
                Kb[:n, n] = e
                Kb[n, :n] = e
                K = Kb
                self.bordered = True
        self.s_r, self.s_c = equilibrate(K)
        Kt = self.s_r[:, None] * K * self.s_c[None, :]
        LU, perm = lu_factor(Kt)
        self.X = lu_inverse(LU, perm)

    def apply(self, r_p: np.ndarray) -> np.ndarray:
        if self.bordered:
            r_p = np.concatenate([r_p, [0.0]])
        d = self.s_c * (self.X @ (self.s_r * r_p))
        return d[:len(self.dofs)]


def partition_weights(patches, n: int) -> np.ndarray:
    """Theta: each unknown weighted by the reciprocal of its patch count (Eq. additive_cav_saddle),
    so that sum_i R_i^T Theta_i R_i = I."""
    count = np.zeros(n)
    for p in patches:
        count[p] += 1.0
    if np.any(count == 0):
        raise ValueError("patch family does not cover every unknown")
    return 1.0 / count


def remove_mean_pressure(w: np.ndarray, N: int) -> np.ndarray:
    """After each sweep the mean pressure is removed (Sec. 3.3)."""
    w = w.copy()
    p = w[2 * N * N:]
    p -= p.mean()
    return w


def additive_sweep(KE, solvers, theta, w, b, N, alpha=1.0):
    """One sweep of the weighted additive CAV relaxation (Eq. additive_cav_saddle):
    r = b - K_E w;  w <- w + alpha sum_i R_i^T Theta_i K_{E,i}^-1 R_i r;  remove mean pressure."""
    r = b - KE @ w
    corr = np.zeros_like(w)
    for s in solvers:
        corr[s.dofs] += theta[s.dofs] * s.apply(r[s.dofs])
    return remove_mean_pressure(w + alpha * corr, N)


def multiplicative_sweep(KE, solvers, w, b, N, inject=None, KE_csc=None):
    """One multiplicative Schwarz sweep in the given patch order (Sec. 3.3):
    r <- b - K_E w; for each p: delta = K_{E,p}^-1 R_p r, w += R_p^T delta, r -= K_E R_p^T delta.
    `inject[p]` (optional) lists the slots of patch p that receive the correction
    (restricted injection for box patches)."""
    KEc = KE.tocsc() if KE_csc is None else KE_csc
    w = w.copy()
    r = b - KE @ w
    for pi, s in enumerate(solvers):
        d = s.apply(r[s.dofs])
        dofs = s.dofs
        if inject is not None:
            slots = inject[pi]
            d = d[slots]
            dofs = dofs[slots]
        w[dofs] += d
        r -= KEc[:, dofs] @ d
    return remove_mean_pressure(w, N)
