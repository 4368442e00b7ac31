"""Pins of the oracle's local solves, transfers, V-cycle and FGMRES:
LU identities, exact whole-domain patches, R = P^T/4 and constant/linear reproduction
(Sec. 4), exact preconditioning, agreement with a dense direct solve, and the paper's
printed FGMRES iteration counts (Sec. 5.1, Table 2)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import ib_workloads as W
from oracle import fgmres, grid, ib, multigrid, patches, smoother


def test_equilibration_is_power_of_two_and_normalises():
    rng = np.random.default_rng(2)
    K = rng.standard_normal((9, 9)) * np.logspace(-6, 6, 9)[:, None]
    s_r, s_c = smoother.equilibrate(K)
    for s in np.concatenate([s_r, s_c]):
        m, e = math.frexp(s)
        assert m == 0.5
    Kt = s_r[:, None] * K * s_c[None, :]
    assert np.all(np.abs(Kt).max(0) <= 1.0) and np.all(np.abs(Kt).max(0) >= 0.5)
    assert np.all(np.abs(s_r[:, None] * K).max(1) >= 0.5)


def test_lu_partial_pivoting_identities():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((12, 12))
    LU, perm = smoother.lu_factor(A)
    L = np.tril(LU, -1) + np.eye(12)
    U = np.triu(LU)
    assert np.allclose(L @ U, A[perm], atol=1e-13)
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0)
    X = smoother.lu_inverse(LU, perm)
    assert np.allclose(X @ A, np.eye(12), atol=1e-12)
    # ties go to the first maximal row
    B = np.array([[1.0, 2.0], [-1.0, 3.0]])
    _, pb = smoother.lu_factor(B)
    assert pb.tolist() == [0, 1]


def _system_levels(sysm, **kw):
    return multigrid.build_hierarchy(sysm, 8, **kw)


def test_whole_domain_patch_solves_exactly():
    # a single patch holding every unknown (bordered for the pressure gauge) makes one
    # additive sweep with Theta = I and alpha = 1 an exact solve
    s = W.target_circle(8, 24, 1e3, 1e-2)
    EE, _ = ib.eulerian_elasticity(s)
    K = grid.reduced_operator(8, s.h, s.rho, s.dt, s.mu, EE)
    n = K.shape[0]
    solver = smoother.PatchSolver(K, np.arange(n), 64, 128)
    assert solver.bordered
    b = s.rhs()
    w = smoother.additive_sweep(K, [solver], np.ones(n), np.zeros(n), b, 8, 1.0)
    assert np.linalg.norm(b - K @ w) <= 1e-12 * np.linalg.norm(b)
    w2 = smoother.multiplicative_sweep(K, [solver], np.zeros(n), b, 8)
    assert np.linalg.norm(b - K @ w2) <= 1e-12 * np.linalg.norm(b)


def test_patch_inverse_times_local_matrix_is_identity():
    s = W.membrane_ellipse(16, 1e4)
    lev = _system_levels(s, factor=False)[0]
    big = max(lev.patches, key=len)
    sol = smoother.PatchSolver(lev.KE, big)
    K = smoother.local_matrix(lev.KE, big)
    Kt = sol.s_r[:, None] * K * sol.s_c[None, :]
    cond = np.linalg.cond(Kt)
    assert np.abs(sol.X @ Kt - np.eye(len(big))).max() <= 50 * cond * np.finfo(float).eps


def test_partition_of_unity():
    s = W.membrane_ellipse(16, 1e4)
    lev = _system_levels(s)[0]
    acc = np.zeros(3 * 16 * 16)
    for p in lev.patches:
        acc[p] += lev.theta[p]
    assert np.allclose(acc, 1.0, atol=1e-15)


def test_transfers():
    Nc = 8
    Pv = multigrid.prolong_velocity(Nc)
    Rv = multigrid.restrict_velocity(Nc)
    assert np.array_equal(Rv.toarray(), 0.25 * Pv.T.toarray())
    assert np.allclose(Rv @ np.ones(2 * 4 * Nc * Nc), 1.0)      # R preserves constants (Sec. 4)
    assert np.allclose(Pv @ np.ones(2 * Nc * Nc), 1.0)
    Pp = multigrid.prolong_pressure(Nc)
    Rp = multigrid.restrict_pressure(Nc)
    assert np.allclose(Pp @ np.ones(Nc * Nc), 1.0) and np.allclose(Rp @ np.ones(4 * Nc * Nc), 1.0)
    # RT0 reproduces u linear in x (interior faces), bilinear reproduces linear p (interior)
    H, h = 1.0 / Nc, 0.5 / Nc
    J, I = np.divmod(np.arange(Nc * Nc), Nc)
    uc = 1.0 + 2.0 * I * H
    uf = (Pv @ np.concatenate([uc, np.zeros(Nc * Nc)]))[:4 * Nc * Nc]
    j, i = np.divmod(np.arange(4 * Nc * Nc), 2 * Nc)
    inner = (i >= 1) & (i <= 2 * Nc - 2)
    assert np.allclose(uf[inner], (1.0 + 2.0 * i * h)[inner])
    pc = 0.5 + 3.0 * (I + 0.5) * H - 1.0 * (J + 0.5) * H
    pf = Pp @ pc
    inner = (i >= 1) & (i <= 2 * Nc - 2) & (j >= 1) & (j <= 2 * Nc - 2)
    assert np.allclose(pf[inner], (0.5 + 3.0 * (i + 0.5) * h - 1.0 * (j + 0.5) * h)[inner])


def test_galerkin_elasticity_symmetric_nsd():
    s = W.membrane_ellipse(16, 1e4)
    EE, pat = ib.eulerian_elasticity(s)
    Ec, pc = multigrid.galerkin_elasticity(EE, pat, 8)
    D = Ec.toarray()
    sc = np.abs(D).max()
    assert np.allclose(D, D.T, atol=1e-13 * sc)
    assert np.linalg.eigvalsh(0.5 * (D + D.T)).max() <= 1e-10 * sc
    assert (pc != pc.T).nnz == 0


def test_coarse_bordered_solve():
    s = W.target_circle(8, 24, 1e3, 1e-2)
    lev = _system_levels(s)[-1]
    b = s.rhs()
    z = multigrid.coarse_solve(lev, b)
    assert np.linalg.norm(b - lev.KE @ z) <= 1e-11 * np.linalg.norm(b)
    assert abs(z[128:].sum()) <= 1e-10 * np.abs(z).max()


def test_fgmres_exact_preconditioner_one_iteration():
    s = W.target_circle(16, 48, 1e3, 1e-2)
    levels = _system_levels(s, factor=False)
    K = levels[0].KE
    inv = multigrid.bordered_inverse(K, 16)
    b = s.rhs()
    x, info = fgmres.fgmres(lambda v: K @ v, b, lambda r: (inv @ np.append(r, 0.0))[:-1],
                            rtol=1e-10, maxit=10)
    assert info["iters"] == 1 and info["relres_true"] <= 1e-10


@pytest.mark.parametrize("mode,nu,alpha", [("multiplicative", 1, 1.0), ("additive", 2, 0.85)])
def test_fgmres_matches_direct_solve(mode, nu, alpha):
    s = W.target_circle(16, 48, 1e3, 1e-2)
    levels = _system_levels(s)
    K = levels[0].KE
    b = s.rhs()
    x, info = fgmres.fgmres(lambda v: K @ v, b,
                            lambda r: multigrid.vcycle(levels, r, nu, nu, mode, alpha),
                            rtol=1e-12, maxit=100)
    assert info["converged"]
    inv = multigrid.bordered_inverse(K, 16)
    xd = (inv @ np.append(b, 0.0))[:-1]
    xd[512:] -= xd[512:].mean()
    x[512:] -= x[512:].mean()
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    # the Givens estimate tracks the true residual
    assert info["relres_true"] <= 10 * max(info["relres_est"], 1e-14)


# Paper's Table 2 / Sec. 5.1 counts for multiplicative CAV, the box smoother B(4,2) with
# restricted injection (target points; its beam counts are a recorded deviation) and
# unpreconditioned FGMRES.
# Marker placement, time level and the right-hand side's source are only partly stated,
# so the pin allows +-3 iterations.
PAPER_COUNTS = [
    ("membrane", 16, "cav", 9),
    ("target", 32, "cav", 10),
    ("target", 32, "none", 19),
    ("beam", 32, "cav", 9),
    ("target", 32, "box", 8),
    ("target", 64, "box", 10),
]


@pytest.mark.parametrize("law,N,prec,want", PAPER_COUNTS)
def test_paper_iteration_counts(law, N, prec, want):
    s = {"membrane": W.paper_membrane, "target": W.paper_target_rows, "beam": W.paper_beam}[law](N)
    b = ib.first_step_rhs(s)
    if prec == "none":
        K = multigrid.build_hierarchy(s, 8, factor=False)[0].KE
        _, info = fgmres.fgmres(lambda v: K @ v, b, lambda r: r, rtol=1e-10, maxit=150, ref="r0")
    else:
        levels = multigrid.build_hierarchy(s, 8, prec)
        K = levels[0].KE
        _, info = fgmres.fgmres(lambda v: K @ v, b,
                                lambda r: multigrid.vcycle(levels, r, 1, 1, "multiplicative"),
                                rtol=1e-10, maxit=150, ref="r0")
    assert info["converged"]
    assert abs(info["iters"] - want) <= 3, info["iters"]


def test_paper_beam_unpreconditioned_fails():
    # Table 2: unpreconditioned FGMRES does not reach 1e-10 within 150 iterations (beam)
    s = W.paper_beam(32)
    K = multigrid.build_hierarchy(s, 8, factor=False)[0].KE
    _, info = fgmres.fgmres(lambda v: K @ v, ib.first_step_rhs(s), lambda r: r, rtol=1e-10,
                            maxit=150, ref="r0")
    assert not info["converged"]


def test_pressure_prolongation_keeps_the_mean():
    # bilinear prolongation on the periodic grid: every coarse cell hands out weights
    # 4 x 9/16 + 8 x 3/16 + 4 x 1/16 = 4 over its four children and their neighbours, so the
    # fine mean equals the coarse mean (a column sum of exactly 4, independent of the field)
    Nc = 8
    Pp = multigrid.prolong_pressure(Nc)
    assert np.allclose(np.asarray(Pp.sum(axis=0)).ravel(), 4.0)
    pc = np.random.default_rng(3).standard_normal(Nc * Nc)
    assert abs((Pp @ pc).mean() - pc.mean()) <= 1e-14


@pytest.mark.parametrize("pre,post,mode", [(2, 0, "additive"), (0, 1, "additive"), (1, 1, "coloured"),
                                           ([0, 2], [1, 2], ["coloured", "additive"]),
                                           ([1, 2], [0, 2], ["coloured", "additive"])])
def test_vcycle_output_pressure_is_mean_free(pre, post, mode):
    # every sweep ends by removing the mean pressure (Sec. 3.3), the bordered coarsest solve
    # returns a mean-free pressure and prolongation keeps the mean, so the cycle's output is
    # mean-free whichever side the finest level's sweeps sit on
    s = W.membrane_ellipse(32, 1e4)
    levels = multigrid.build_hierarchy(s, 8, "cav")
    b = s.rhs()
    z = multigrid.vcycle(levels, b, pre, post, mode, 0.85)
    p = z[2 * 32 * 32:]
    assert np.abs(p).max() > 0.0
    assert abs(p.mean()) <= 1e-13 * np.abs(p).max()
