"""Colour classes for a parallel ordering of the multiplicative CAV sweep (Sec. 3.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's smoother visits the patches one after another: each patch solve reads the
residual left by all earlier solves (multiplicative Schwarz).  Two patches p and q can be
solved at the same time without changing that result when neither solve reads what the
other writes: the solve of q reads w on every column of K_E in the rows of q and writes w on
the unknowns of q, so p and q are independent exactly when no entry of K_E couples an
unknown of p with an unknown of q (and they share no unknown).  Grouping the patches into
classes of mutually independent patches and visiting the classes in turn is then one
multiplicative sweep whose patch order is "class by class".  This is the parallel route to
the paper's multiplicative smoother; the class order is a reading (the paper uses
lexicographic order, which has no parallelism).

Readings taken here (identical in the CUDA library):
  * coupling is structural: the stencil pattern of the Stokes rows (Sec. 2) plus the
    structural pattern of E_E on that level (the same pattern the CAV sets read);
  * classes come from first-fit greedy colouring, visiting the enlarged patches (more than
    the five unknowns of V_ij) in ascending cell order, then the standard ones in ascending
    cell order; a patch takes the smallest class index not already taken by a coupled
    patch visited before it;
  * inside a class the patches are independent, so their order is immaterial; the sweep
    below visits them in ascending cell order.

The same classes serve the box smoother B(b,o) (Sec. 3.1, 3.3): one patch per b x b block,
every patch larger than five unknowns, so the visit order is the blocks' lexicographic order
(the paper's order for its box sweep).  Its restricted injection writes only the unknowns
of the unexpanded block, a subset of the patch, so two patches that K_E does not couple
stay independent and the conflict relation above is unchanged (it is conservative there).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import grid, smoother


def coupling_pattern(N: int, ee_pattern: sp.spmatrix | None) -> sp.csr_matrix:
    """Boolean structural pattern of K_E on an N x N level, with its diagonal: the Stokes
    blocks [[A0, G], [-D, 0]] (all stencil entries are nonzero for any h, rho/dt > 0) plus
    E_E's structural pattern in the velocity block."""
    K0 = grid.reduced_operator(N, 1.0, 1.0, 1.0, 1.0, None)
    pat = sp.csr_matrix(K0 != 0, dtype=bool)
    n = 3 * N * N
    pat = pat + sp.identity(n, dtype=bool, format="csr")
    if ee_pattern is not None:
        E = sp.csr_matrix(ee_pattern, dtype=bool)
        pat = pat + sp.bmat([[E, None], [None, sp.csr_matrix((N * N, N * N), dtype=bool)]],
                            format="csr", dtype=bool)
    pat = sp.csr_matrix(pat, dtype=bool)
    pat.sort_indices()
    return pat


def visit_order(patches) -> list[int]:
    """Enlarged patches in cell order, then standard patches in cell order."""
    big = [c for c, p in enumerate(patches) if len(p) > 5]
    std = [c for c, p in enumerate(patches) if len(p) <= 5]
    return big + std


def greedy_colours(patches, pattern: sp.csr_matrix) -> np.ndarray:
    """First-fit colour of every patch (indexed by cell) in visit_order."""
    n = pattern.shape[0]
    holders: list[list[int]] = [[] for _ in range(n)]
    for c, p in enumerate(patches):
        for k in p:
            holders[int(k)].append(c)
    colour = np.full(len(patches), -1, dtype=np.int64)
    for c in visit_order(patches):
        reach = np.unique(pattern[patches[c]].indices)
        taken = {int(colour[q]) for k in reach for q in holders[int(k)] if colour[q] >= 0}
        k = 0
        while k in taken:
            k += 1
        colour[c] = k
    return colour


def coloured_sweep(KE, solvers, colours, w, b, N, inject=None):
    """One multiplicative sweep (Sec. 3.3) visiting the colour classes in turn, each class's
    patches in ascending patch order: for each patch p, r_p = b_p - (K_E w)_p from the
    current iterate, delta = K_{E,p}^-1 r_p, w_p += delta; then the mean pressure is removed.
    `inject[p]` (optional) lists the slots of patch p that receive the correction (the
    restricted injection of the box smoother, Sec. 3.3); the other slots' entries of delta
    are dropped."""
    w = np.array(w, dtype=np.float64, copy=True)
    KE = sp.csr_matrix(KE)
    for k in range(int(colours.max()) + 1):
        for c in np.nonzero(colours == k)[0]:
            s = solvers[c]
            r_p = b[s.dofs] - KE[s.dofs] @ w
            d = s.apply(r_p)
            if inject is None:
                w[s.dofs] += d
            else:
                w[s.dofs[inject[c]]] += d[inject[c]]
    return smoother.remove_mean_pressure(w, N)
