"""Pins of the oracle's colour classes and its class-by-class multiplicative sweep (Sec. 3.3).

  * validity, brute force: no two patches of one class are coupled by a nonzero of the
    assembled K_E (numeric entries, physical coefficients) or of E_E's structural pattern;
  * first fit, brute force: every patch's class is the smallest index not taken by a coupled
    patch visited before it;
  * independence: visiting one class's patches in reverse order gives the same bits;
  * the sweep equals the sequential multiplicative sweep of Sec. 3.3 (which the paper's
    printed iteration counts pin) run in the class-by-class patch order;
  * the paper's membrane case converges in a count close to the printed one;
  * the same for the box smoother B(4,2) with restricted injection: valid first-fit classes
    over the blocks, the class-by-class sweep equal to the sequential restricted sweep in
    class order, and the paper's target-point count.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import colouring, fgmres, ib, multigrid, smoother


CASES = [lambda: W.membrane_ellipse(16, 1e4),
         lambda: W.beam_curve(16, 48, 1.0, 10.0),
         lambda: W.target_circle(16, 40, 1e3, 1e-3)]


def _dense_coupling(lev):
    """Coupling read off the assembled operator: numeric nonzeros of K_E, the structural
    pattern of E_E (entries that might cancel numerically still couple), and the diagonal."""
    D = lev.KE.toarray() != 0.0
    NN2 = 2 * lev.N * lev.N
    if lev.pattern is not None:
        D[:NN2, :NN2] |= lev.pattern.toarray()
    np.fill_diagonal(D, True)
    return D


@pytest.mark.parametrize("mk", CASES)
def test_classes_are_independent_and_first_fit(mk):
    _check_classes(multigrid.build_hierarchy(mk(), 8, factor=False))


def test_box_classes_are_independent_and_first_fit():
    # B(4,2) patches (208 unknowns each, one per 4 x 4 block): every patch is "enlarged", so
    # the visit order is the blocks' lexicographic order
    _check_classes(multigrid.build_hierarchy(W.beam_curve(32, 96, 1.0, 10.0), 8, "box", factor=False))


def _check_classes(levels):
    for lev in levels[:-1]:
        col = multigrid.level_colours(lev)
        D = _dense_coupling(lev)
        pats = lev.patches
        n_p = len(pats)
        # brute-force pairwise coupling between all patches
        coupled = np.zeros((n_p, n_p), dtype=bool)
        for a in range(n_p):
            rows = D[pats[a]]
            for b in range(n_p):
                coupled[a, b] = rows[:, pats[b]].any()
        assert np.array_equal(coupled, coupled.T)
        for a in range(n_p):
            same = np.nonzero(col == col[a])[0]
            assert not any(coupled[a, b] for b in same if b != a)
        # first fit in the visit order: enlarged (more than 5 unknowns) then standard,
        # each in ascending cell order
        order = [c for c in range(n_p) if len(pats[c]) > 5] + [c for c in range(n_p) if len(pats[c]) <= 5]
        seen = []
        for c in order:
            taken = {int(col[q]) for q in seen if coupled[c, q]}
            assert int(col[c]) not in taken
            assert set(range(int(col[c]))) <= taken
            seen.append(c)


def test_order_inside_a_class_is_immaterial():
    s = W.membrane_ellipse(16, 1e4)
    lev = multigrid.build_hierarchy(s, 8)[0]
    col = multigrid.level_colours(lev)
    b = s.rhs()
    w0 = np.random.default_rng(3).uniform(-1, 1, b.size)

    def run(reverse):
        w = w0.copy()
        K = lev.KE.tocsr()
        for k in range(int(col.max()) + 1):
            members = list(np.nonzero(col == k)[0])
            if reverse:
                members = members[::-1]
            for c in members:
                sv = lev.solvers[c]
                w[sv.dofs] += sv.apply(b[sv.dofs] - K[sv.dofs] @ w)
        return w

    assert np.array_equal(run(False), run(True))


@pytest.mark.parametrize("mk", CASES[:2])
def test_coloured_sweep_is_the_multiplicative_sweep_in_class_order(mk):
    s = mk()
    levels = multigrid.build_hierarchy(s, 8)
    b = s.rhs()
    for lev in levels[:-1]:
        col = multigrid.level_colours(lev)
        n = 3 * lev.N * lev.N
        bl = b[:n] if n == b.size else np.random.default_rng(lev.N).uniform(-1, 1, n)
        w0 = np.random.default_rng(lev.N + 1).uniform(-1, 1, n)
        order = np.lexsort((np.arange(col.size), col))
        want = smoother.multiplicative_sweep(lev.KE, [lev.solvers[c] for c in order], w0, bl, lev.N)
        got = colouring.coloured_sweep(lev.KE, lev.solvers, col, w0, bl, lev.N)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_box_coloured_sweep_is_the_restricted_multiplicative_sweep_in_class_order():
    # restricted injection (Sec. 3.3): each box patch writes only the unknowns of its
    # unexpanded block; the class-by-class sweep equals the sequential one in class order
    s = W.beam_curve(32, 96, 1.0, 10.0)
    levels = multigrid.build_hierarchy(s, 8, "box")
    b = s.rhs()
    for lev in levels[:-1]:
        col = multigrid.level_colours(lev)
        n = 3 * lev.N * lev.N
        bl = b[:n] if n == b.size else np.random.default_rng(lev.N).uniform(-1, 1, n)
        w0 = np.random.default_rng(lev.N + 1).uniform(-1, 1, n)
        order = np.lexsort((np.arange(col.size), col))
        want = smoother.multiplicative_sweep(lev.KE, [lev.solvers[c] for c in order], w0, bl, lev.N,
                                             [lev.inject[c] for c in order])
        got = colouring.coloured_sweep(lev.KE, lev.solvers, col, w0, bl, lev.N, lev.inject)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
        # the injection is restricted: dropping it changes the result
        full = colouring.coloured_sweep(lev.KE, lev.solvers, col, w0, bl, lev.N)
        assert np.linalg.norm(full - got) > 1e-3 * np.linalg.norm(got)


def test_paper_target_box_count_with_class_order():
    # Sec. 5.2: B(4,2) takes 8 FGMRES iterations on the target-point rows at N = 32 with its
    # lexicographic sweep; the class-by-class order is another multiplicative ordering
    s = W.paper_target_rows(32)
    levels = multigrid.build_hierarchy(s, 8, "box")
    K = levels[0].KE
    _, info = fgmres.fgmres(lambda v: K @ v, ib.first_step_rhs(s),
                            lambda r: multigrid.vcycle(levels, r, 1, 1, "coloured"),
                            rtol=1e-10, maxit=150, ref="r0")
    assert info["converged"]
    assert abs(info["iters"] - 8) <= 3, info["iters"]


def test_whole_domain_single_class_is_exact():
    s = W.target_circle(8, 24, 1e3, 1e-2)
    EE, _ = ib.eulerian_elasticity(s)
    from oracle import grid
    K = grid.reduced_operator(8, s.h, s.rho, s.dt, s.mu, EE)
    n = K.shape[0]
    sv = smoother.PatchSolver(K, np.arange(n), 64, 128)
    b = s.rhs()
    w = colouring.coloured_sweep(K, [sv], np.zeros(1, dtype=np.int64), np.zeros(n), b, 8)
    assert np.linalg.norm(b - K @ w) <= 1e-12 * np.linalg.norm(b)


def test_paper_membrane_count_with_class_order():
    # Sec. 5.1: 9 FGMRES iterations for the membrane at N = 16 with the lexicographic
    # multiplicative sweep; the class-by-class order is another multiplicative ordering
    s = W.paper_membrane(16)
    levels = multigrid.build_hierarchy(s, 8)
    K = levels[0].KE
    _, info = fgmres.fgmres(lambda v: K @ v, ib.first_step_rhs(s),
                            lambda r: multigrid.vcycle(levels, r, 1, 1, "coloured"),
                            rtol=1e-10, maxit=150, ref="r0")
    assert info["converged"]
    assert abs(info["iters"] - 9) <= 3, info["iters"]


def _round_bf16(a):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((u >> np.uint32(16)) & np.uint32(1)) + np.uint32(0x7FFF)
    return ((u + r) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)


def test_bf16_rounded_inverses_make_the_undamped_sweep_diverge():
    # why the library refuses BF16 inverses for the multiplicative smoother: with the
    # enlarged patches' inverses rounded to 8 bits, one class-by-class sweep increases the
    # residual by many orders of magnitude, while FP32 rounding leaves it contracting
    s = W.membrane_ellipse(32, 1e4)
    lev = multigrid.build_hierarchy(s, 8)[0]
    col = multigrid.level_colours(lev)
    b = s.rhs()
    r0 = np.linalg.norm(b)
    X64 = [sv.X for sv in lev.solvers]
    for sv in lev.solvers:
        if len(sv.dofs) > 5:
            sv.X = np.asarray(sv.X, dtype=np.float32).astype(np.float64)
    w = colouring.coloured_sweep(lev.KE, lev.solvers, col, np.zeros(b.size), b, lev.N)
    assert np.linalg.norm(b - lev.KE @ w) < r0
    for sv, X in zip(lev.solvers, X64):
        if len(sv.dofs) > 5:
            sv.X = _round_bf16(X)
    w = colouring.coloured_sweep(lev.KE, lev.solvers, col, np.zeros(b.size), b, lev.N)
    assert np.linalg.norm(b - lev.KE @ w) > 1e6 * r0
