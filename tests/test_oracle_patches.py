"""Pins of the oracle's patch families (Sec. 3) against literal re-statements of the set
definitions on a dense boolean pattern, and against the special cases the paper names:
B(1,0) is the standard Vanka family, and CAV returns V_ij wherever U^_ij = U_ij (so with
no structure CAV is Vanka)."""
import numpy as np
import pytest
import scipy.sparse as sp

import ib_workloads as W
from oracle import ib, multigrid, patches


def _literal_cav(N, dense_pat):
    """Eq. (cav_patch_set) written out with Python sets over a dense boolean matrix."""
    NN = N * N

    def u(i, j):
        return (j % N) * N + (i % N)

    def v(i, j):
        return NN + (j % N) * N + (i % N)

    def p(i, j):
        return 2 * NN + (j % N) * N + (i % N)

    def V(i, j):
        return {p(i, j), u(i, j), u(i + 1, j), v(i, j), v(i, j + 1)}

    def C(k):
        if k < NN:
            j, i = divmod(k, N)
            return {((i - 1) % N, j), (i, j)}
        j, i = divmod(k - NN, N)
        return {(i, (j - 1) % N), (i, j)}

    out = []
    for j in range(N):
        for i in range(N):
            Uij = {u(i, j), u(i + 1, j), v(i, j), v(i, j + 1)}
            Uhat = set(Uij)
            for l in Uij:
                Uhat |= set(np.nonzero(dense_pat[:, l])[0].tolist())
                Uhat |= set(np.nonzero(dense_pat[l, :])[0].tolist())
            if Uhat == Uij:
                out.append(sorted(V(i, j)))
            else:
                cells = set()
                for k in Uhat:
                    cells |= C(k)
                dofs = set()
                for (a, b) in cells:
                    dofs |= V(a, b)
                out.append(sorted(dofs))
    return out


@pytest.mark.parametrize("mk", [lambda: W.target_circle(16, 40, 1e3, 1e-3),
                                lambda: W.membrane_ellipse(16, 1e4),
                                lambda: W.beam_curve(16, 48, 1.0, 10.0),
                                lambda: W.paper_target_rows(16)])
def test_cav_matches_literal_definition(mk):
    s = mk()
    _, pat = ib.eulerian_elasticity(s)
    got = patches.cav_patches(s.N, pat)
    want = _literal_cav(s.N, pat.toarray())
    assert len(got) == len(want) == s.N ** 2
    for g, w in zip(got, want):
        assert g.tolist() == w


def test_cav_on_galerkin_level_matches_literal_definition():
    s = W.membrane_ellipse(32, 1e4)
    EE, pat = ib.eulerian_elasticity(s)
    _, pc = multigrid.galerkin_elasticity(EE, pat, 16)
    got = patches.cav_patches(16, pc)
    want = _literal_cav(16, pc.toarray())
    assert all(g.tolist() == w for g, w in zip(got, want))


def test_cav_without_structure_is_vanka():
    N = 8
    empty = sp.csr_matrix((2 * N * N, 2 * N * N), dtype=bool)
    got = patches.cav_patches(N, empty)
    ref = patches.vanka_patches(N)
    assert all(np.array_equal(a, b) for a, b in zip(got, ref))
    assert all(len(a) == 5 for a in got)


def test_box_1_0_is_vanka():
    N = 8
    box = patches.box_patches(N, 1, 0)
    ref = patches.vanka_patches(N)
    assert all(np.array_equal(a, r) and np.array_equal(b, r) for (a, b), r in zip(box, ref))


def test_box_4_2_sizes():
    # B(4,2): 8x8 expanded cell blocks -> 64 pressures + 2*8*9 faces = 208 unknowns each
    N = 16
    box = patches.box_patches(N, 4, 2)
    assert len(box) == (N // 4) ** 2
    assert all(len(p) == 64 + 2 * 8 * 9 for p, _ in box)
    assert all(len(b) == 16 + 2 * 4 * 5 for _, b in box)


def test_box_4_2_order_and_geometry():
    # Sec. 3.1/3.3: blocks in lexicographic order of their lower-left cells (i fastest); the
    # patch holds the pressures of the cells within o layers of the block (periodic), the
    # injected set those of the block itself, and every velocity of a held cell
    N, b, o = 16, 4, 2
    NN = N * N
    for p, (patch, block) in enumerate(patches.box_patches(N, b, o)):
        I, J = (p % (N // b)) * b, (p // (N // b)) * b
        pres = patch[patch >= 2 * NN] - 2 * NN
        want = sorted(c for c in range(NN)
                      if ((c % N - I + o) % N) < b + 2 * o and ((c // N - J + o) % N) < b + 2 * o)
        assert list(pres) == want
        bp = block[block >= 2 * NN] - 2 * NN
        assert list(bp) == sorted(c for c in range(NN) if ((c % N - I) % N) < b and ((c // N - J) % N) < b)
        assert set(block) <= set(patch)
        # each held cell's four faces are held
        for c in pres:
            i, j = c % N, c // N
            for k in (j * N + i, j * N + (i + 1) % N, NN + j * N + i, NN + ((j + 1) % N) * N + i):
                assert k in set(patch)


def test_cav_patches_contain_their_vanka_patch_and_cover():
    s = W.membrane_ellipse(16, 1e4)
    _, pat = ib.eulerian_elasticity(s)
    got = patches.cav_patches(s.N, pat)
    ref = patches.vanka_patches(s.N)
    for g, r in zip(got, ref):
        assert set(r.tolist()) <= set(g.tolist())
    assert any(len(g) > 5 for g in got)
