"""Newton's method for one semi-implicit time step with a nonlinear force law (Sec. 5.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The backward-Euler step of Eqs. im_disc_mom and im_disc_advec with the Lagrangian force taken
at the updated configuration and spreading / interpolation at the start of the step:

    rho/dt (u - u^n) - mu L u + G p = S^n F(X^n + dt J^n u) + f,     -D u = 0,

with X^{n+1} = X^n + dt J^n u.  Newton's method on w = (u, p) linearises F at
X_k = X^n + dt J^n u_k; its Jacobian is K_E of Eq. Eul_schur with E_E = S^n E(X_k) J^n, E the
force's tangent dF/dX (the paper's statement that Newton produces the Eulerian system with E
replaced by the tangent).  Solving for the next iterate directly,

    K_E(X_k) w_{k+1} = [ rho/dt u^n + f + S^n (F(X_k) - dt E(X_k) J^n u_k) ; 0 ].

The linear systems are solved here by a direct factorisation of the bordered matrix
[[K_E, e], [e^T, 0]] (e the pressure indicator: the restriction to mean-zero pressure, Sec. 2),
the plain definition of the solve that the CAV-preconditioned FGMRES approximates.  The
iteration stops when the nonlinear residual falls below rtol relative to its first value or
below atol (the paper's test with 1e-8 for both).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import grid, ib


def _force_and_tangent(sysm, X):
    """F(X) and E(X) = dF/dX of the record's law at the configuration X, component-major."""
    s = replace(sysm, X=X, meta={**sysm.meta, "X_lin": X})
    return ib.force_vector(s), ib.elasticity(s)[0]


def _solve_bordered(K, rhs, N):
    n = K.shape[0]
    e = np.zeros(n)
    e[2 * N * N:] = 1.0
    B = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
    return spla.spsolve(B, np.concatenate([rhs, [0.0]]))[:n]


def residual(sysm, u_n, f, w):
    """R(w) = [rho/dt u + (-mu L u) + G p - rho/dt u^n - f - S^n F(X^n + dt J^n u); -D u]."""
    N, h = sysm.N, sysm.h
    NN2 = 2 * N * N
    K0 = grid.reduced_operator(N, h, sysm.rho, sysm.dt, sysm.mu, None)
    S = ib.spreading_matrix(N, h, sysm.X, sysm.omega)
    J = ib.interpolation_matrix(N, h, sysm.X)
    X = _cm_to_xy(_xy_to_cm(sysm.X) + sysm.dt * (J @ w[:NN2]))
    F, _ = _force_and_tangent(sysm, X)
    R = K0 @ w
    R[:NN2] -= sysm.rho / sysm.dt * u_n + f + S @ F
    return R


def _xy_to_cm(X):
    return np.concatenate([X[:, 0], X[:, 1]])


def _cm_to_xy(x):
    M = x.size // 2
    return np.stack([x[:M], x[M:]], 1)


def cav_fgmres_solver(mode="coloured", nu=1, alpha=1.0, rtol=1e-9, maxit=150, coarsest_N=8):
    """A linear solver for newton_step as the paper runs it (Sec. 5.3): the CAV hierarchy
    rebuilt for each Newton system, right-preconditioned FGMRES to rtol relative to ||r_0||
    with one V-cycle per iteration.  Records the iteration counts in its `iters` list."""
    from . import fgmres, multigrid

    def solve(sys_k, K, rhs):
        levels = multigrid.build_hierarchy(sys_k, coarsest_N, "cav")
        x, info = fgmres.fgmres(lambda v: K @ v, rhs,
                                lambda r: multigrid.vcycle(levels, r, nu, nu, mode, alpha),
                                rtol=rtol, maxit=maxit, ref="r0")
        solve.iters.append(info["iters"])
        return x

    solve.iters = []
    return solve


def newton_step(sysm, u_n=None, f=None, w0=None, rtol=1e-8, atol=1e-8, maxit=20, linear_solve=None):
    """One time step from (X^n = sysm.X, u^n) by Newton's method.  Returns (w, X^{n+1},
    history of ||R|| per iterate, number of Newton corrections).  `linear_solve(sys_k, K, rhs)`
    (default: the bordered direct solve) solves each Newton system; sys_k is the record with
    its linearisation point at X_k."""
    N, h = sysm.N, sysm.h
    NN2 = 2 * N * N
    n = 3 * N * N
    u_n = np.zeros(NN2) if u_n is None else u_n
    f = np.zeros(NN2) if f is None else f
    w = np.zeros(n) if w0 is None else np.array(w0, dtype=np.float64)
    S = ib.spreading_matrix(N, h, sysm.X, sysm.omega)
    J = ib.interpolation_matrix(N, h, sysm.X)
    Xn = _xy_to_cm(sysm.X)
    hist = [np.linalg.norm(residual(sysm, u_n, f, w))]
    k = 0
    while k < maxit and hist[-1] > max(rtol * hist[0], atol):
        Xk = _cm_to_xy(Xn + sysm.dt * (J @ w[:NN2]))
        F, E = _force_and_tangent(sysm, Xk)
        EE = (S @ E @ J).tocsr()
        K = grid.reduced_operator(N, h, sysm.rho, sysm.dt, sysm.mu, EE)
        rhs = np.zeros(n)
        rhs[:NN2] = sysm.rho / sysm.dt * u_n + f + S @ (F - sysm.dt * (E @ (J @ w[:NN2])))
        if linear_solve is None:
            w = _solve_bordered(K, rhs, N)
        else:
            w = linear_solve(replace(sysm, meta={**sysm.meta, "X_lin": Xk}), K, rhs)
        k += 1
        hist.append(np.linalg.norm(residual(sysm, u_n, f, w)))
    X_next = _cm_to_xy(Xn + sysm.dt * (J @ w[:NN2]))
    return w, X_next, hist, k
