"""Geometric multigrid of Sec. 4.

  * hierarchy by halving the cell count per direction; level 0 is the finest grid here
    (the paper counts l_max down to 0), coarsened while N_l / 2 >= the coarsest size;
  * velocity prolongation P: lowest-order Raviart-Thomas interpolation -- a fine face on a
    coarse face takes that coarse value, a fine face on a coarse cell's midline takes the
    mean of the cell's two coarse faces of that component; restriction R = (1/4) P^T;
  * pressure: bilinear prolongation between cell centres (weights 9/16, 3/16, 3/16, 1/16),
    restriction by averaging the four fine cells;
  * A0, D, G rediscretised with h_l; E_E^(l-1) = R E_E^(l) P (Galerkin), whose structural
    pattern is the boolean product pattern (reading);
  * patches and local factorisations on every level but the coarsest, which is solved by a
    precomputed direct factorisation of the bordered system [[K_E, e], [e^T, 0]] (e = the
    pressure indicator: the restriction to U_h x P_h of Sec. 2);
  * V-cycle: nu_pre sweeps, residual restriction, recursive coarse correction, prolongation,
    nu_post sweeps (one and one in the paper).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import colouring, grid, ib, patches as patchmod, smoother
from .grid import U, V


def prolong_velocity(Nc: int) -> sp.csr_matrix:
    """RT0 prolongation from the Nc grid to the 2Nc grid (both components)."""
    Nf = 2 * Nc
    rows, cols, vals = [], [], []
    for j in range(Nf):
        for i in range(Nf):
            # u face (i, j)
            r = grid.idx(Nf, U, i, j)
            if i % 2 == 0:
                rows.append(r); cols.append(grid.idx(Nc, U, i // 2, j // 2)); vals.append(1.0)
            else:
                for I in ((i - 1) // 2, (i + 1) // 2):
                    rows.append(r); cols.append(grid.idx(Nc, U, I, j // 2)); vals.append(0.5)
            # v face (i, j)
            r = grid.idx(Nf, V, i, j)
            if j % 2 == 0:
                rows.append(r); cols.append(grid.idx(Nc, V, i // 2, j // 2)); vals.append(1.0)
            else:
                for J in ((j - 1) // 2, (j + 1) // 2):
                    rows.append(r); cols.append(grid.idx(Nc, V, i // 2, J)); vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * Nf * Nf, 2 * Nc * Nc))


def restrict_velocity(Nc: int) -> sp.csr_matrix:
    """R = P* = (1/4) P^T."""
    return (0.25 * prolong_velocity(Nc).T).tocsr()


def prolong_pressure(Nc: int) -> sp.csr_matrix:
    """Bilinear interpolation between cell centres, Nc -> 2Nc (pressure block only)."""
    Nf = 2 * Nc
    rows, cols, vals = [], [], []
    for j in range(Nf):
        J0, sj = j // 2, (-1 if j % 2 == 0 else 1)
        for i in range(Nf):
            I0, si = i // 2, (-1 if i % 2 == 0 else 1)
            r = j * Nf + i
            for (dI, dJ, w) in ((0, 0, 9 / 16), (si, 0, 3 / 16), (0, sj, 3 / 16), (si, sj, 1 / 16)):
                rows.append(r); cols.append(((J0 + dJ) % Nc) * Nc + (I0 + dI) % Nc); vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(Nf * Nf, Nc * Nc))


def restrict_pressure(Nc: int) -> sp.csr_matrix:
    """Cell averaging of the four fine cells of each coarse cell."""
    Nf = 2 * Nc
    rows, cols, vals = [], [], []
    for J in range(Nc):
        for I in range(Nc):
            for b in (0, 1):
                for a in (0, 1):
                    rows.append(J * Nc + I); cols.append((2 * J + b) * Nf + 2 * I + a); vals.append(0.25)
    return sp.csr_matrix((vals, (rows, cols)), shape=(Nc * Nc, Nf * Nf))


def prolong(Nc: int) -> sp.csr_matrix:
    return sp.block_diag([prolong_velocity(Nc), prolong_pressure(Nc)], format="csr")


def restrict(Nc: int) -> sp.csr_matrix:
    return sp.block_diag([restrict_velocity(Nc), restrict_pressure(Nc)], format="csr")


def galerkin_elasticity(EE_f: sp.csr_matrix, pat_f: sp.csr_matrix, Nc: int):
    """E_E^(l-1) = R E_E^(l) P and its structural pattern (boolean product)."""
    Pv = prolong_velocity(Nc)
    Rv = 0.25 * Pv.T
    EE_c = (Rv @ EE_f @ Pv).tocsr()
    Pb = Pv.copy()
    Pb.data = np.ones_like(Pb.data)
    Pb = Pb.astype(np.int64)
    pat = (Pb.T @ pat_f.astype(np.int64) @ Pb).tocsr()
    pat.data = np.ones_like(pat.data)
    pat = pat.astype(bool)
    return ib.pattern_values(pat, EE_c), pat


@dataclass
class Level:
    N: int
    h: float
    KE: sp.csr_matrix
    EE: sp.csr_matrix | None
    pattern: sp.csr_matrix | None
    patches: list = field(default_factory=list)
    inject: list | None = None
    solvers: list = field(default_factory=list)
    theta: np.ndarray | None = None
    coarse_inverse: np.ndarray | None = None
    KE_csc: sp.csc_matrix | None = None
    colours: np.ndarray | None = None


def level_colours(lev: Level) -> np.ndarray:
    """Colour classes of the level's patches (computed on first use)."""
    if lev.colours is None:
        lev.colours = colouring.greedy_colours(lev.patches, colouring.coupling_pattern(lev.N, lev.pattern))
    return lev.colours


def level_sizes(N: int, coarsest_N: int = 8) -> list[int]:
    sizes = [N]
    while sizes[-1] // 2 >= coarsest_N and sizes[-1] % 2 == 0:
        sizes.append(sizes[-1] // 2)
    return sizes


def build_hierarchy(sysm, coarsest_N: int = 8, kind: str = "cav", box=(4, 2),
                    factor: bool = True, with_structure: bool = True) -> list[Level]:
    """Levels from finest to coarsest, with patches and factorisations (Sec. 4)."""
    sizes = level_sizes(sysm.N, coarsest_N)
    if with_structure and sysm.M > 0:
        EE, pat = ib.eulerian_elasticity(sysm)
    else:
        EE, pat = None, None
    levels = []
    for li, N in enumerate(sizes):
        if li > 0 and EE is not None:
            EE, pat = galerkin_elasticity(EE, pat, N)
        h = sysm.L / N
        KE = grid.reduced_operator(N, h, sysm.rho, sysm.dt, sysm.mu, EE)
        lev = Level(N=N, h=h, KE=KE, EE=EE, pattern=pat)
        last = li == len(sizes) - 1
        if last:
            lev.coarse_inverse = bordered_inverse(KE, N)
        else:
            if kind == "cav":
                lev.patches = patchmod.cav_patches(N, pat)
            elif kind == "vanka":
                lev.patches = patchmod.vanka_patches(N)
            elif kind == "box":
                pairs = patchmod.box_patches(N, *box)
                lev.patches = [p for p, _ in pairs]
                lev.inject = [np.nonzero(np.isin(p, blk))[0] for p, blk in pairs]
            else:
                raise ValueError(kind)
            if factor:
                lev.solvers = [smoother.PatchSolver(KE, p, N * N, 2 * N * N) for p in lev.patches]
                lev.theta = smoother.partition_weights(lev.patches, 3 * N * N)
                lev.KE_csc = KE.tocsc()
        levels.append(lev)
    return levels


def bordered_inverse(KE: sp.csr_matrix, N: int) -> np.ndarray:
    """Dense inverse of [[K_E, e], [e^T, 0]] by LU with partial pivoting (coarsest level)."""
    n = KE.shape[0]
    K = np.zeros((n + 1, n + 1))
    K[:n, :n] = KE.toarray()
    K[2 * N * N:n, n] = 1.0
    K[n, 2 * N * N:n] = 1.0
    LU, perm = smoother.lu_factor(K)
    return smoother.lu_inverse(LU, perm)


def coarse_solve(lev: Level, r: np.ndarray) -> np.ndarray:
    return (lev.coarse_inverse @ np.concatenate([r, [0.0]]))[:-1]


def sweep(lev: Level, w, b, mode: str = "additive", alpha: float = 1.0):
    if mode == "additive":
        return smoother.additive_sweep(lev.KE, lev.solvers, lev.theta, w, b, lev.N, alpha)
    if mode == "coloured":
        return colouring.coloured_sweep(lev.KE, lev.solvers, level_colours(lev), w, b, lev.N, lev.inject)
    return smoother.multiplicative_sweep(lev.KE, lev.solvers, w, b, lev.N, lev.inject, lev.KE_csc)


def vcycle(levels, b, nu_pre=1, nu_post=1, mode="additive",
           alpha: float = 1.0, li: int = 0, trace: list | None = None) -> np.ndarray:
    """z = B b: one V-cycle with zero initial guess (Sec. 4).  nu_pre, nu_post and mode may be
    per-level lists (smoothing levels, finest first).  `trace`, if given, collects
    (level, stage, vector) after every sweep for step-by-step comparison."""
    lev = levels[li]
    if isinstance(mode, (list, tuple)):
        return _vcycle_levels(levels, b, nu_pre, nu_post, mode, alpha, li, trace)
    if li == len(levels) - 1:
        z = coarse_solve(lev, b)
        if trace is not None:
            trace.append((li, "coarse", z.copy()))
        return z
    x = np.zeros_like(b)
    for s in range(nu_pre):
        x = sweep(lev, x, b, mode, alpha)
        if trace is not None:
            trace.append((li, f"pre{s}", x.copy()))
    r = b - lev.KE @ x
    Nc = levels[li + 1].N
    bc = restrict(Nc) @ r
    xc = vcycle(levels, bc, nu_pre, nu_post, mode, alpha, li + 1, trace)
    x = x + prolong(Nc) @ xc
    if trace is not None:
        trace.append((li, "prolonged", x.copy()))
    for s in range(nu_post):
        x = sweep(lev, x, b, mode, alpha)
        if trace is not None:
            trace.append((li, f"post{s}", x.copy()))
    return x


def _vcycle_levels(levels, b, nu_pre, nu_post, mode, alpha, li, trace):
    """The V-cycle with level li's own smoother mode[li] and sweep counts."""
    lev = levels[li]
    if li == len(levels) - 1:
        z = coarse_solve(lev, b)
        if trace is not None:
            trace.append((li, "coarse", z.copy()))
        return z
    x = np.zeros_like(b)
    for s in range(nu_pre[li]):
        x = sweep(lev, x, b, mode[li], alpha)
        if trace is not None:
            trace.append((li, f"pre{s}", x.copy()))
    r = b - lev.KE @ x
    Nc = levels[li + 1].N
    xc = _vcycle_levels(levels, restrict(Nc) @ r, nu_pre, nu_post, mode, alpha, li + 1, trace)
    x = x + prolong(Nc) @ xc
    if trace is not None:
        trace.append((li, "prolonged", x.copy()))
    for s in range(nu_post[li]):
        x = sweep(lev, x, b, mode[li], alpha)
        if trace is not None:
            trace.append((li, f"post{s}", x.copy()))
    return x
