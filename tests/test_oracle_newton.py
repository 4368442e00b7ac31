"""Pins of the oracle's Newton iteration for one semi-implicit step (Sec. 5.3).

  * a linear force law makes the step's equations affine in w: Newton stops after one
    correction, whose iterate is the single linear solve of K_E w = b with the step's
    right-hand side of Eq. Eul_schur (the pinned operators and right-hand side);
  * the fiber law converges superlinearly (each residual drop far larger than the one before,
    which a wrong tangent would turn into a linear rate) to the paper's 1e-8 test within the
    two or so corrections per step the paper reports for its fiber;
  * the converged state satisfies the nonlinear step equations and X^{n+1} = X^n + dt J^n u.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import ib_workloads as W
from oracle import grid, ib, newton


def _bordered_solve(K, b, N):
    n = K.shape[0]
    e = np.zeros(n)
    e[2 * N * N:] = 1.0
    B = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
    return spla.spsolve(B, np.concatenate([b, [0.0]]))[:n]


def test_linear_law_takes_one_correction_equal_to_the_linear_solve():
    s = W.membrane_ellipse(16, 1e4)
    un = 0.1 * W.uniform_pm1(11, 2 * s.N ** 2)
    w, _, hist, k = newton.newton_step(s, u_n=un)
    assert k == 1 and hist[1] <= 1e-12 * hist[0]
    EE, _ = ib.eulerian_elasticity(s)
    K = grid.reduced_operator(s.N, s.h, s.rho, s.dt, s.mu, EE)
    want = _bordered_solve(K, ib.step_rhs(s, u_prev=un), s.N)
    assert np.linalg.norm(w - want) <= 1e-10 * np.linalg.norm(want)


def test_fiber_newton_converges_superlinearly():
    s = W.fiber_periodic(16)
    for un in (None, 0.05 * W.uniform_pm1(12, 2 * s.N ** 2)):
        w, X1, hist, k = newton.newton_step(s, u_n=un)
        assert 1 <= k <= 3 and hist[-1] <= max(1e-8 * hist[0], 1e-8), hist
        assert hist[1] < hist[0]
        for a in range(1, len(hist) - 1):
            assert hist[a + 1] / hist[a] <= 0.1 * hist[a] / hist[a - 1], hist
        # the step equations hold at the converged iterate, and the markers moved with J u
        assert np.linalg.norm(newton.residual(s, np.zeros(2 * s.N ** 2) if un is None else un,
                                              np.zeros(2 * s.N ** 2), w)) == hist[-1]
        J = ib.interpolation_matrix(s.N, s.h, s.X)
        U = J @ w[:2 * s.N ** 2]
        assert np.allclose(X1, s.X + s.dt * np.stack([U[:s.M], U[s.M:]], 1), rtol=0, atol=1e-15)


def test_fiber_newton_with_cav_fgmres_matches_the_papers_counts():
    # Sec. 5.3, N = 16: Newton needs about two corrections per step and FGMRES (CAV V-cycle,
    # one multiplicative sweep per side, hierarchy rebuilt per Newton system, 1e-9) 8.65
    # iterations per solve on average, 13 at most; the stand-in's first step from a bent
    # fiber lands within those bounds (its set-up is periodic, not the paper's channel)
    s = W.fiber_periodic(16)
    sol = newton.cav_fgmres_solver(mode="multiplicative")
    w, _, hist, k = newton.newton_step(s, linear_solve=sol)
    assert k <= 3 and hist[-1] <= 1e-8 * hist[0]
    assert all(abs(i - 8.65) <= 3 and i <= 13 for i in sol.iters), sol.iters
    w_direct, _, _, _ = newton.newton_step(s)
    assert np.linalg.norm(w - w_direct) <= 1e-6 * np.linalg.norm(w_direct)
