"""Patch families of Sec. 3: standard Vanka, box B(b,o) and coupling-aware Vanka (CAV).

  U_{ij} = {u_{ij}, u_{i+1,j}, v_{ij}, v_{i,j+1}},   V_{ij} = {p_{ij}} u U_{ij}      (Sec. 3.1)
  V(C)   = union of V_c over the cells c in C                                        (Sec. 3.1)
  B(b,o): block with lower-left cell (i,j) -> cells (i+r, j+s), -o <= r,s <= b+o-1    (Sec. 3.1)
  C(u_{ij}) = {(i-1,j), (i,j)},  C(v_{ij}) = {(i,j-1), (i,j)}                         (Sec. 3.2)
  U^_{ij} = U_{ij} u {k : (E_E)_{kl} != 0 or (E_E)_{lk} != 0 for some l in U_{ij}}   (Sec. 3.2)
  V^CAV_{ij} = V_{ij} if U^_{ij} = U_{ij}, else V(C(U^_{ij}))                         (Eq. cav_patch_set)

Every patch is a sorted array of global indices (u block, then v, then p; index j N + i
inside a block).  One CAV patch per cell, cells in lexicographic order c = j N + i
(i fastest) -- the paper says "lexicographic" without naming the axis order; this is
the reading taken.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import U, V, P, idx


def velocity_set(N: int, i: int, j: int) -> list[int]:
    """U_{ij}."""
    return [int(idx(N, U, i, j)), int(idx(N, U, i + 1, j)),
            int(idx(N, V, i, j)), int(idx(N, V, i, j + 1))]


def vanka_set(N: int, i: int, j: int) -> set[int]:
    """V_{ij}."""
    return {int(idx(N, P, i, j))} | set(velocity_set(N, i, j))


def union_patch(N: int, cells) -> np.ndarray:
    """V(C) as a sorted index array."""
    out: set[int] = set()
    for (i, j) in cells:
        out |= vanka_set(N, i, j)
    return np.array(sorted(out), dtype=np.int64)


def incident_cells(N: int, k: int) -> list[tuple[int, int]]:
    """C(k) for a velocity index k."""
    c, rem = divmod(k, N * N)
    j, i = divmod(rem, N)
    if c == U:
        return [((i - 1) % N, j), (i, j)]
    if c == V:
        return [(i, (j - 1) % N), (i, j)]
    raise ValueError("C is defined on velocity unknowns only")


def vanka_patches(N: int) -> list[np.ndarray]:
    """B(1,0): the standard family, one patch per cell in lexicographic order."""
    return [union_patch(N, [(c % N, c // N)]) for c in range(N * N)]


def box_patches(N: int, b: int, o: int):
    """B(b,o) patches in lexicographic order of the blocks' lower-left cells, with the
    unexpanded block's unknowns V(block) for restricted injection (Sec. 3.3)."""
    out = []
    for J in range(0, N, b):
        for I in range(0, N, b):
            cells = [((I + r) % N, (J + s) % N) for s in range(-o, b + o) for r in range(-o, b + o)]
            block = [((I + r) % N, (J + s) % N) for s in range(b) for r in range(b)]
            out.append((union_patch(N, cells), union_patch(N, block)))
    return out


def cav_patches(N: int, pattern: sp.spmatrix | None) -> list[np.ndarray]:
    """Eq. (cav_patch_set) for every cell; `pattern` is the boolean pattern of E_E (2N^2 square)
    on this level, or None when there is no structure."""
    if pattern is None:
        return vanka_patches(N)
    Pr = sp.csr_matrix(pattern, dtype=bool)
    Pc = Pr.T.tocsr()  # (E_E)_{kl} != 0 read along column l
    out = []
    for c in range(N * N):
        i, j = c % N, c // N
        Uij = velocity_set(N, i, j)
        Uhat = set(Uij)
        for l in Uij:
            Uhat.update(Pr.indices[Pr.indptr[l]:Pr.indptr[l + 1]].tolist())
            Uhat.update(Pc.indices[Pc.indptr[l]:Pc.indptr[l + 1]].tolist())
        if Uhat == set(Uij):
            out.append(union_patch(N, [(i, j)]))
        else:
            cells = set()
            for k in Uhat:
                cells.update(incident_cells(N, k))
            out.append(union_patch(N, sorted(cells)))
    return out


def patch_stats(patches) -> dict:
    n = np.array([len(p) for p in patches], dtype=np.int64)
    distinct = len({p.tobytes() for p in patches})
    return {"count": int(n.size), "sum_n": int(n.sum()), "sum_n2": int((n * n).sum()),
            "max_n": int(n.max()) if n.size else 0, "mean_n": float(n.mean()) if n.size else 0.0,
            "enlarged": int((n > 5).sum()), "distinct": distinct}
