"""Immersed-boundary coupling operators (Sec. 2) and Lagrangian force matrices (Sec. 2, 5.1, 5.2).

  delta_h(x) = h^-2 phi(x/h) phi(y/h) with Peskin's four-point phi (cited in Sec. 2);
  f = S F:  f^u_{ij} = sum_k F^x_k delta_h(x_{i-1/2,j} - X_k) omega_k  (and v likewise);
  U = J u:  U^x_k   = sum_{ij} u_{ij} delta_h(x_{i-1/2,j} - X_k) h^2;
  E_E = S E J (Eq. intro_saddle).

Lagrangian vectors are ordered component-major: index c M + k, c in {0: x, 1: y}.

Readings where the paper is silent:
  * phi is the standard four-point kernel
      |r| <= 1:      (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8
      1 <= |r| <= 2: (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8
      otherwise 0.
  * A marker couples to face index i along one axis iff |i - t| < 2 with t = X/h - offset
    (offset 0 where the face sits on grid lines, 1/2 where it sits at cell centres).
    This is the structural support: E_E's nonzero pattern (used by CAV, Eq. cav_patch_set)
    is the boolean product of the supports of S, E and J, never a test of computed values.
    The support is evaluated with the fixed IEEE sequence
      q = X / h;  t = q - offset;  f = floor(t);  a = t - f;  r_s = (a + 1) - s, s = 0..3
    with index f - 1 + s in the support iff |r_s| < 2.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .grid import U, V


def phi(r):
    """Peskin's four-point kernel (peskin2002, the kernel named in Sec. 2)."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    a = r <= 1.0
    b = (r > 1.0) & (r < 2.0)
    out[a] = (3.0 - 2.0 * r[a] + np.sqrt(1.0 + 4.0 * r[a] - 4.0 * r[a] ** 2)) / 8.0
    out[b] = (5.0 - 2.0 * r[b] - np.sqrt(-7.0 + 12.0 * r[b] - 4.0 * r[b] ** 2)) / 8.0
    return out


def axis_support(x: float, h: float, offset: float):
    """Face indices (unwrapped) along one axis coupled to a marker at coordinate x, with their
    1-D weights phi(i + offset - x/h).  Returns (indices, weights), each of length <= 4."""
    q = x / h
    t = q - offset
    f = math.floor(t)
    a = t - f
    idxs, wts = [], []
    for s in range(4):
        r = (a + 1.0) - s
        if abs(r) < 2.0:
            idxs.append(int(f) - 1 + s)
            wts.append(float(phi(r)))
    return idxs, wts


# Position of the two velocity components within a cell: (x offset, y offset) in units of h.
FACE_OFFSET = {U: (0.0, 0.5), V: (0.5, 0.0)}


def interpolation_matrix(N: int, h: float, X: np.ndarray) -> sp.csr_matrix:
    """J (2M x 2N^2): U_k = sum_ij u_ij phi phi (the h^-2 of delta_h cancels the h^2)."""
    M = X.shape[0]
    rows, cols, vals = [], [], []
    for c in (U, V):
        ox, oy = FACE_OFFSET[c]
        for k in range(M):
            ix, wx = axis_support(X[k, 0], h, ox)
            iy, wy = axis_support(X[k, 1], h, oy)
            for jj, wyj in zip(iy, wy):
                for ii, wxi in zip(ix, wx):
                    rows.append(c * M + k)
                    cols.append(c * N * N + (jj % N) * N + (ii % N))
                    vals.append(wxi * wyj)
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * M, 2 * N * N))


def support_pattern(N: int, h: float, X: np.ndarray) -> sp.csr_matrix:
    """Structural pattern of J as a 0/1 integer matrix."""
    Jm = interpolation_matrix(N, h, X)
    B = Jm.copy()
    B.data = np.ones_like(B.data)
    return B.astype(np.int64)


def spreading_matrix(N: int, h: float, X: np.ndarray, omega: np.ndarray) -> sp.csr_matrix:
    """S (2N^2 x 2M): f_face = sum_k F_k phi phi omega_k / h^2."""
    Jm = interpolation_matrix(N, h, X)
    M = X.shape[0]
    W = sp.diags(np.concatenate([omega, omega]) / h ** 2)
    return (Jm.T @ W).tocsr() if M else sp.csr_matrix((2 * N * N, 0))


def _cyclic(M: int, stencil: dict) -> sp.csr_matrix:
    rows, cols, vals = [], [], []
    for k in range(M):
        for d, c in stencil.items():
            rows.append(k)
            cols.append((k + d) % M)
            vals.append(c)
    return sp.csr_matrix((vals, (rows, cols)), shape=(M, M))


def force_matrix(law: int, M: int, ds: float, k_target: float, k_stretch: float,
                 k_bend: float) -> sp.csr_matrix:
    """Lagrangian elasticity matrix E (2M x 2M), identical on the x and y components.

    target   (Sec. 5.2):  F_k = kappa_t (X_target - X_k)      ->  E = -kappa_t I
    membrane (Eq. disc_force_law): F_k = kappa_s/ds^2 (X_{k+1} + X_{k-1} - 2 X_k)
    beam     (Sec. 5.2):  F = -kappa_b d^4X/ds^4, centred five-point stencil / ds^4,
                          plus the membrane term when kappa_s != 0 (both on a closed curve).
    """
    if law == 0:
        E1 = -k_target * sp.identity(M, format="csr")
    else:
        # tethers (-k_target I, Sec. 5.2) may accompany the membrane and beam laws
        st = {}
        if k_stretch != 0.0:
            c = k_stretch / ds ** 2
            for d, w in ((-1, 1.0), (0, -2.0), (1, 1.0)):
                st[d] = st.get(d, 0.0) + c * w
        if law == 2 and k_bend != 0.0:
            c = -k_bend / ds ** 4
            for d, w in ((-2, 1.0), (-1, -4.0), (0, 6.0), (1, -4.0), (2, 1.0)):
                st[d] = st.get(d, 0.0) + c * w
        if k_target != 0.0:
            st[0] = st.get(0, 0.0) - k_target
        E1 = _cyclic(M, st)
    return sp.block_diag([E1, E1], format="csr")


def force_pattern(law: int, M: int, k_stretch: float, k_bend: float,
                  k_target: float = 0.0) -> sp.csr_matrix:
    """Structural pattern of E: the stencil offsets whose coefficient is nonzero."""
    if law == 0:
        offs = [0]
    else:
        offs = set()
        if k_stretch != 0.0:
            offs |= {-1, 0, 1}
        if law == 2 and k_bend != 0.0:
            offs |= {-2, -1, 0, 1, 2}
        if k_target != 0.0:
            offs |= {0}
        offs = sorted(offs)
    B1 = _cyclic(M, {d: 1 for d in offs})
    B1.data = np.ones_like(B1.data)
    return sp.block_diag([B1, B1], format="csr").astype(np.int64)


LAW_FIBER = 3


def fiber_params(sysm):
    """The fiber law's parameters (Sec. 5.3) from a workload record: EI = k_bend, K_s =
    k_stretch, K_p, K_t and the clamp point X_c from its meta fields."""
    from . import fiber
    return fiber.FiberParams(M=sysm.M, ds=sysm.ds, EI=sysm.k_bend, K_s=sysm.k_stretch,
                             K_p=sysm.meta["k_pos"], K_t=sysm.meta["k_tan"], X_c=tuple(sysm.meta["X_c"]))


def fiber_linearisation_point(sysm):
    """Where the fiber's force and tangent are taken: the Newton iterate X_lin when the record
    carries one, else X (S and J always stay at X, Sec. 5.3)."""
    Xl = sysm.meta.get("X_lin")
    return sysm.X if Xl is None else np.asarray(Xl, dtype=np.float64)


def elasticity(sysm):
    """E of the record's law at its configuration: the linear laws' matrix, or the fiber's
    Newton tangent dF/dX at X (Sec. 5.3), with its structural pattern."""
    if sysm.law == LAW_FIBER:
        from . import fiber
        p = fiber_params(sysm)
        return fiber.tangent(p, fiber_linearisation_point(sysm)), fiber.tangent_pattern(p).astype(np.int64)
    E = force_matrix(sysm.law, sysm.M, sysm.ds, sysm.k_target, sysm.k_stretch, sysm.k_bend)
    return E, force_pattern(sysm.law, sysm.M, sysm.k_stretch, sysm.k_bend, sysm.k_target)


def eulerian_elasticity(sysm):
    """E_E = S E J (values) and its structural pattern (bool CSR), for a workload record."""
    N, h = sysm.N, sysm.h
    S = spreading_matrix(N, h, sysm.X, sysm.omega)
    J = interpolation_matrix(N, h, sysm.X)
    E, Eb = elasticity(sysm)
    EE = (S @ E @ J).tocsr()
    Jb = support_pattern(N, h, sysm.X)
    pat = (Jb.T @ Eb @ Jb).tocsr()
    pat.data = np.ones_like(pat.data)
    pat = pat.astype(bool)
    # carry the values on exactly the structural pattern (explicit zeros kept)
    EE = pattern_values(pat, EE)
    return EE, pat


def pattern_values(pat: sp.csr_matrix, A: sp.spmatrix) -> sp.csr_matrix:
    """CSR with the sparsity of `pat` and the values of A at those positions."""
    pat = pat.tocsr()
    pat.sort_indices()
    A = A.tocsr()
    rows = np.repeat(np.arange(pat.shape[0]), np.diff(pat.indptr))
    vals = np.asarray(A[rows, pat.indices]).ravel() if pat.nnz else np.zeros(0)
    return sp.csr_matrix((vals, pat.indices.copy(), pat.indptr.copy()), shape=pat.shape)


def first_step_rhs(sysm) -> np.ndarray:
    """Right-hand side of Eq. (Eul_schur) for the first backward Euler step from rest (Sec. 5):
    u^n = 0 so b = 0 and the velocity rows carry S E X^n; the target law's source term
    kappa_t X_target^{n+1} (Sec. 5.2) is added to E X^n.  Pressure rows are zero."""
    N, h = sysm.N, sysm.h
    S = spreading_matrix(N, h, sysm.X, sysm.omega)
    F = force_vector(sysm)
    b = np.zeros(3 * N * N)
    b[:2 * N * N] = S @ F
    return b


def force_vector(sysm) -> np.ndarray:
    """F = E X^n + k_target X_target (component-major): the linear laws' force at X^n
    (Eq. disc_force_law, Sec. 5.2); the fiber's nonlinear force F(X^n) (Sec. 5.3)."""
    if sysm.law == LAW_FIBER:
        from . import fiber
        return fiber.force(fiber_params(sysm), fiber_linearisation_point(sysm))
    E = force_matrix(sysm.law, sysm.M, sysm.ds, sysm.k_target, sysm.k_stretch, sysm.k_bend)
    F = E @ np.concatenate([sysm.X[:, 0], sysm.X[:, 1]])
    if sysm.k_target != 0.0 and sysm.X_target is not None:
        F = F + sysm.k_target * np.concatenate([sysm.X_target[:, 0], sysm.X_target[:, 1]])
    return F


def step_rhs(sysm, u_prev=None, f_body=None) -> np.ndarray:
    """Right-hand side of Eq. (Eul_schur) for one semi-implicit step without convection:
    velocity rows (rho/dt) u^n + f_body + S (E X^n + k_target X_target), pressure rows 0."""
    N, h = sysm.N, sysm.h
    S = spreading_matrix(N, h, sysm.X, sysm.omega)
    b = np.zeros(3 * N * N)
    b[:2 * N * N] = S @ force_vector(sysm)
    if u_prev is not None:
        b[:2 * N * N] += (sysm.rho / sysm.dt) * u_prev[:2 * N * N]
    if f_body is not None:
        b[:2 * N * N] += f_body
    return b


def advect(sysm, u) -> np.ndarray:
    """X^{n+1} = X^n + dt J^n u^{n+1} (Eq. im_disc_advec), returned as (M, 2)."""
    J = interpolation_matrix(sysm.N, sysm.h, sysm.X)
    U = J @ u[:2 * sysm.N * sysm.N]
    M = sysm.M
    return sysm.X + sysm.dt * np.stack([U[:M], U[M:]], axis=1)
