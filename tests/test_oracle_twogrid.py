"""Pins of the oracle's two-grid spectrum routine (Sec. 5.1, Table 1):

  * with an exact preconditioner on U_h x P_h (the bordered direct inverse) B K is the identity
    there: rho(T) = 0 and every |lambda| = 1;
  * for the membrane two-grid cycle, rho(T) from the eigenvalues equals the asymptotic
    contraction factor of the stationary iteration e <- (I - B K) e measured by power iteration
    (mean pressure projected out, as the subspace requires).
"""
import numpy as np

import ib_workloads as W
from oracle import grid, ib, multigrid, twogrid


def test_mean_zero_basis():
    N = 4
    Q = twogrid.mean_zero_basis(N)
    assert Q.shape == (48, 47)
    assert np.allclose(Q.T @ Q, np.eye(47), atol=1e-14)
    c = np.zeros(48)
    c[32:] = 1.0
    assert np.abs(Q.T @ c).max() < 1e-14


def test_exact_preconditioner_gives_zero_radius():
    s = W.target_circle(8, 24, 1e3, 1e-2)
    EE, _ = ib.eulerian_elasticity(s)
    K = grid.reduced_operator(8, s.h, s.rho, s.dt, s.mu, EE)
    Kinv = multigrid.bordered_inverse(K, 8)
    n = K.shape[0]
    BK = twogrid.preconditioned_operator(lambda v: K @ v, lambda r: (Kinv @ np.concatenate([r, [0.0]]))[:-1], n)
    summ = twogrid.spectrum_summary(BK, 8)
    assert summ["rho_T"] < 1e-9
    assert abs(summ["min_abs_lambda"] - 1.0) < 1e-9 and abs(summ["max_abs_lambda"] - 1.0) < 1e-9


def test_radius_matches_power_iteration():
    s = W.paper_membrane(16, 1e6)
    levels = multigrid.build_hierarchy(s, 8)
    assert len(levels) == 2
    K = levels[0].KE
    n = K.shape[0]
    BK = twogrid.preconditioned_operator(lambda v: K @ v, lambda r: multigrid.vcycle(levels, r, 1, 1, "coloured"), n)
    rho = twogrid.spectrum_summary(BK, 16)["rho_T"]
    e = np.random.default_rng(1).standard_normal(n)
    for _ in range(80):
        e[2 * 256:] -= e[2 * 256:].mean()
        e2 = e - BK @ e
        ratio = np.linalg.norm(e2) / np.linalg.norm(e)
        e = e2 / np.linalg.norm(e2)
    assert abs(ratio - rho) <= 1e-3 * rho, (ratio, rho)
