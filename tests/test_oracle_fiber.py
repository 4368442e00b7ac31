"""Pins of the oracle's nonlinear fiber law (Sec. 5.3): energies, force and Newton tangent.

  * the gradient equals central differences of the energy, and the Hessian central
    differences of the gradient, at bent and stretched configurations;
  * bending and stretching are invariant under translations and rotations: their internal
    force sums to zero and does no work along an infinitesimal rotation, and their energy
    is unchanged by a finite rotation;
  * at the straight reference configuration of spacing ds the force vanishes, and the
    tangent reduces to the textbook linearisations: -(K_s/ds^2) (open second difference)
    on x, -(EI/ds^4) (open fourth difference, D2^T D2) on y, no x-y coupling;
  * the clamp terms vanish at the prescribed midpoint position and tangent;
  * the paper's marker counts (13, 25, 49, 97 at N = 16 ... 128);
  * the structural pattern holds every nonzero of the tangent.
"""
import numpy as np
import pytest

from oracle import fiber


def _params(M=11, ds=0.05, K_p=3.0, K_t=0.7):
    return fiber.FiberParams(M=M, ds=ds, EI=0.02, K_s=40.0, K_p=K_p, K_t=K_t, X_c=(1.0, 1.5))


def _bent(p, seed=0, amp=0.25):
    rng = np.random.default_rng(seed)
    X = fiber.straight_fiber(p.M, p.ds, p.X_c)
    return X + amp * p.ds * rng.standard_normal(X.shape)


def _cmv(X):
    return np.concatenate([X[:, 0], X[:, 1]])


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_and_hessian_match_finite_differences(seed):
    p = _params()
    x = _cmv(_bent(p, seed))
    g = fiber.gradient(p, x)
    H = fiber.hessian(p, x).toarray()
    eps = 1e-6 * p.ds
    g_fd = np.zeros_like(x)
    H_fd = np.zeros_like(H)
    for i in range(x.size):
        e = np.zeros_like(x)
        e[i] = eps
        g_fd[i] = (fiber.energy(p, x + e)["total"] - fiber.energy(p, x - e)["total"]) / (2 * eps)
        H_fd[:, i] = (fiber.gradient(p, x + e) - fiber.gradient(p, x - e)) / (2 * eps)
    assert np.linalg.norm(g - g_fd) <= 1e-6 * np.linalg.norm(g)
    assert np.linalg.norm(H - H_fd) <= 1e-6 * np.linalg.norm(H)
    assert np.abs(H - H.T).max() <= 1e-13 * np.abs(H).max()


def test_internal_forces_are_translation_and_rotation_free():
    p = _params(K_p=0.0, K_t=0.0)
    X = _bent(p, 3, amp=0.4)
    x = _cmv(X)
    F = fiber.force(p, x)
    M = p.M
    scale = np.abs(F).max()
    assert abs(F[:M].sum()) <= 1e-12 * scale * M and abs(F[M:].sum()) <= 1e-12 * scale * M
    # no work along the rotation generator (-y, x) about any point
    rot = np.concatenate([-(X[:, 1] - 0.3), X[:, 0] + 0.2])
    assert abs(F @ rot) <= 1e-12 * scale * np.abs(rot).sum()
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    E0 = fiber.energy(p, X)
    E1 = fiber.energy(p, X @ R.T + np.array([0.3, -0.1]))
    for k in ("bend", "stretch"):
        assert abs(E1[k] - E0[k]) <= 1e-11 * E0[k]
    # the translation modes are in the tangent's null space
    T = fiber.tangent(p, x).toarray()
    ones = np.concatenate([np.ones(M), np.zeros(M)])
    assert np.abs(T @ ones).max() <= 1e-10 * np.abs(T).max()


def test_straight_reference_linearises_to_second_and_fourth_differences():
    p = _params(K_p=0.0, K_t=0.0)
    M, ds = p.M, p.ds
    X = fiber.straight_fiber(M, ds, p.X_c)
    x = _cmv(X)
    assert np.abs(fiber.force(p, x)).max() <= 1e-9 * p.K_s
    T = fiber.tangent(p, x).toarray()
    D1 = np.diff(np.eye(M), axis=0)          # (M-1) x M first difference
    D2 = np.diff(np.eye(M), n=2, axis=0)     # (M-2) x M second difference
    want_xx = -(p.K_s / ds ** 2) * (D1.T @ D1)
    want_yy = -(p.EI / ds ** 4) * (D2.T @ D2)
    scale = max(np.abs(want_xx).max(), np.abs(want_yy).max())
    assert np.abs(T[:M, :M] - want_xx).max() <= 1e-12 * scale
    assert np.abs(T[M:, M:] - want_yy).max() <= 1e-12 * scale
    assert np.abs(T[:M, M:]).max() <= 1e-12 * scale
    # interior rows of the y block are the beam stencil -(EI/ds^4) [1, -4, 6, -4, 1]
    mid = M // 2
    assert np.allclose(T[M + mid, M + mid - 2:M + mid + 3] * ds ** 4 / -p.EI, [1, -4, 6, -4, 1], rtol=1e-12)


def test_clamp_terms_vanish_at_the_prescribed_midpoint():
    p = _params()
    X = fiber.straight_fiber(p.M, p.ds, p.X_c)
    E = fiber.energy(p, X)
    assert E["position"] == 0.0 and E["tangent"] <= 1e-28 and E["total"] <= 1e-20
    # moving the midpoint costs K_p/2 |d|^2 exactly
    Y = X.copy()
    Y[p.m] += [0.01, -0.02]
    assert np.isclose(fiber.energy(p, Y)["position"], 0.5 * p.K_p * 5e-4, rtol=1e-12)


def test_paper_marker_counts_and_parameters():
    # Sec. 5.3: 13, 25, 49 and 97 fiber markers at N = 16, 32, 64, 128; K_s = 375 at N = 64
    for N, M in ((16, 13), (32, 25), (64, 49), (128, 97)):
        p = fiber.paper_params(N)
        assert p.M == M and p.M % 2 == 1
        assert np.isclose((p.M - 1) * p.ds, 0.375)
    p = fiber.paper_params(64)
    assert (p.K_s, p.K_p, p.K_t) == (375.0, 1200.0, 7.03125)
    assert fiber.paper_params(128).K_s == 750.0


def test_pattern_holds_every_nonzero():
    p = _params()
    pat = fiber.tangent_pattern(p).toarray()
    for seed in range(3):
        T = fiber.tangent(p, _cmv(_bent(p, seed))).toarray()
        assert not np.any((T != 0) & ~pat)


def test_fiber_eulerian_elasticity_couples_components_and_is_symmetric():
    import ib_workloads as W
    from oracle import ib
    s = W.fiber_periodic(16)
    EE, pat = ib.eulerian_elasticity(s)
    NN = s.N ** 2
    A = EE.toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.abs(A[:NN, NN:]).max() > 1e-3 * np.abs(A).max()   # u-v coupling through the tangent
    assert not np.any((A != 0) & ~pat.toarray())


@pytest.mark.parametrize("N,avg,mx", [(16, 11.76, 201), (32, 7.85, 198), (64, 6.36, 195)])
def test_paper_fiber_patch_sizes(N, avg, mx):
    # Sec. 5.3, the fiber refinement table: average and largest CAV patch on the finest level
    # (the paper's averages run over a simulation, this is one bent configuration with the
    # paper's marker count, spacing and stiffnesses): within 15 % and 25 %
    import ib_workloads as W
    from oracle import ib, patches
    s = W.fiber_periodic(N)
    _, pat = ib.eulerian_elasticity(s)
    sz = np.array([len(p) for p in patches.cav_patches(s.N, pat)])
    assert abs(sz.mean() - avg) <= 0.15 * avg, sz.mean()
    assert abs(sz.max() - mx) <= 0.25 * mx, sz.max()
