"""The coloured multiplicative smoother at full size (the bench's membrane, N = 256, and the
membrane at N = 128, kappa_s = 1e2), checked through properties that hold at any size, since
the oracle's class-by-class sweep is too slow there:

  * colour classes (GPU export): no two patches of a class share an unknown or are coupled by
    a structural entry of K_E (coupling read off the oracle's assembled K_E and E_E pattern, as
    the sparse product P C P^T of the patch incidence P and the coupling C), and each patch's
    class is the smallest one not taken by a coupled patch visited before it (first fit);
  * after one GPU sweep (FP64 inverses) every terminal patch -- one coupled to no patch of a
    later class -- has a zero local residual: nothing after its own solve changed its rows.  Tolerance 1000 cond eps of the
    larger of the local residual before the sweep and the local right-hand side, cond the
    patch inverse's condition number (the local solve is exact in exact arithmetic, and the
    residual it starts from is the one the sweep left, not the initial one);
  * the FGMRES solve with FP32 inverses reaches 1e-10 (true residual from the oracle's K_E).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import ib_workloads as W
from oracle import multigrid as omg, smoother as osm
from tests.gpu_helpers import gpu_hierarchy, host, torch_dev

pytestmark = pytest.mark.gpu

CASES = {"membrane256": lambda: W.config2(256, 1e4), "membrane128_k1e2": lambda: W.config2(128, 1e2)}


class Full:
    pass


@pytest.fixture(scope="module", params=sorted(CASES))
def full(request):
    F = Full()
    F.name, F.rec = request.param, CASES[request.param]()
    F.levels = omg.build_hierarchy(F.rec, 8, "cav", factor=False)
    F.sys, F.h64 = gpu_hierarchy(F.rec, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, precision="fp64",
                                 smoother="coloured")
    return F


def _coupled_patches(lev, off, dofs):
    n = 3 * lev.N * lev.N
    C = sp.csr_matrix(lev.KE != 0, dtype=np.int32)
    if lev.pattern is not None:
        E = sp.csr_matrix(lev.pattern, dtype=np.int32)
        C = C + sp.bmat([[E, None], [None, sp.csr_matrix((lev.N ** 2, lev.N ** 2), dtype=np.int32)]],
                        format="csr")
    C = (C + sp.identity(n, dtype=np.int32, format="csr")).astype(bool).astype(np.int32)
    n_p = off.size - 1
    P = sp.csr_matrix((np.ones(dofs.size, dtype=np.int32), dofs, off), shape=(n_p, n))
    M = (P @ C @ P.T).tocsr()
    M.data[:] = 1
    return M


def test_full_colour_classes_valid_and_first_fit(full):
    from paper_2608_14310_b300 import api
    for l, lev in enumerate(full.levels[:-1]):
        off, dofs = api.cav_patch_export(full.h64, l)
        col = api.cav_colour_export(full.h64, l).astype(np.int64)
        M = _coupled_patches(lev, off, dofs)
        rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
        cols = M.indices
        off_diag = rows != cols
        assert not np.any(col[rows[off_diag]] == col[cols[off_diag]]), f"level {l}: coupled patches share a class"
        sizes = np.diff(off)
        order = np.concatenate([np.nonzero(sizes > 5)[0], np.nonzero(sizes <= 5)[0]])
        rank = np.empty_like(order)
        rank[order] = np.arange(order.size)
        for p in range(M.shape[0]):
            nb = M.indices[M.indptr[p]:M.indptr[p + 1]]
            earlier = nb[rank[nb] < rank[p]]
            taken = set(col[earlier].tolist())
            assert col[p] not in taken and taken >= set(range(int(col[p]))), (l, p)
        print(f"{full.name} level {l}: {int(col.max()) + 1} classes valid over {M.shape[0]} patches")


def test_full_terminal_patch_residuals_vanish(full):
    from paper_2608_14310_b300 import api
    lev = full.levels[0]
    NN = lev.N ** 2
    off, dofs = api.cav_patch_export(full.h64, 0)
    col = api.cav_colour_export(full.h64, 0).astype(np.int64)
    M = _coupled_patches(lev, off, dofs)
    later = np.zeros(M.shape[0], dtype=bool)
    rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    np.logical_or.at(later, rows, col[M.indices] > col[rows])
    terminal = np.nonzero(~later)[0]
    sizes = np.diff(off)
    # the enlarged terminal patches first (the sampled set), then a few standard ones
    last = np.concatenate([terminal[sizes[terminal] > 5][:20], terminal[sizes[terminal] <= 5][:4]])
    rng = np.random.default_rng(41)
    b = rng.uniform(-1, 1, 3 * NN)
    b[2 * NN:] -= b[2 * NN:].mean()
    w0 = rng.uniform(-1, 1, 3 * NN) * 1e-3
    w = torch_dev(w0)
    api.cav_sweep(full.h64, 0, torch_dev(b), w)
    got = host(w)
    r_before = b - lev.KE @ w0
    r_after = b - lev.KE @ got
    worst = 0.0
    for p in last[:24]:
        d = dofs[off[p]:off[p + 1]].astype(np.int64)
        sol = osm.PatchSolver(lev.KE, d, NN, 2 * NN)
        cond = np.linalg.cond(sol.X)
        ref = max(np.linalg.norm(r_before[d]), np.linalg.norm(b[d]), 1e-300)
        ratio = np.linalg.norm(r_after[d]) / ref
        bound = 1000 * cond * np.finfo(float).eps
        worst = max(worst, ratio / bound)
        assert ratio <= bound, (p, ratio, cond)
    print(f"{full.name}: {terminal.size} terminal patches, {last.size} checked, local residual ratio "
          f"<= {worst:.2e} of its bound")


def test_full_fgmres_fp32(full):
    from paper_2608_14310_b300 import api
    h32 = api.cav_setup(full.sys, nu_pre=1, nu_post=1, precision="fp32", smoother="coloured")
    b = full.rec.rhs()
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(full.sys, h32, torch_dev(b), x, rtol=1e-10, maxit=150)
    rel = np.linalg.norm(b - full.levels[0].KE @ host(x)) / np.linalg.norm(b)
    assert info["converged"] == 1 and rel <= 2e-10, (info, rel)
    print(f"{full.name}: coloured FP32 {info['iters']} iterations, true relative residual {rel:.2e}")
