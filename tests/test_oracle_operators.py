"""Pins of the oracle's operators against facts fixed independently of its code:
the four-point kernel's moment identities, closed-form Fourier symbols of the MAC
stencils, the adjointness of S and J (Sec. 2), the kernel's exact reproduction of
constant and linear fields, closed-form spectra of the cyclic force laws, and a
brute-force structural pattern of E_E computed from marker-face distances."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import ib_workloads as W
from oracle import grid, ib


def test_phi_moment_identities():
    # Peskin's four-point kernel: sum_j phi(r-j) = 1, even and odd sums 1/2,
    # first moment 0, sum of squares 3/8 -- for every shift r.
    r = np.random.default_rng(1).uniform(-3, 3, 10_000)
    js = np.arange(-6, 7)
    vals = ib.phi(r[:, None] - js[None, :])
    assert np.allclose(vals.sum(1), 1.0, atol=1e-14)
    even = (js % 2 == 0)
    assert np.allclose(vals[:, even].sum(1), 0.5, atol=1e-14)
    assert np.allclose(vals[:, ~even].sum(1), 0.5, atol=1e-14)
    assert np.allclose((vals * (r[:, None] - js[None, :])).sum(1), 0.0, atol=1e-14)
    assert np.allclose((vals ** 2).sum(1), 3.0 / 8.0, atol=1e-14)


def test_phi_special_values():
    assert ib.phi(0.0) == pytest.approx(0.5, abs=1e-16)
    assert ib.phi(1.0) == pytest.approx(0.25, abs=1e-16)
    assert ib.phi(0.5) == pytest.approx((2 + math.sqrt(2)) / 8, abs=1e-16)
    assert ib.phi(1.5) == pytest.approx((2 - math.sqrt(2)) / 8, abs=1e-16)
    assert ib.phi(2.0) == 0.0 and ib.phi(2.5) == 0.0
    assert ib.phi(-0.7) == ib.phi(0.7)


def test_divergence_is_minus_gradient_transpose():
    # Sec. 2: the standard MAC discretisation satisfies D = -G^T (exactly)
    for N in (4, 8, 13):
        h = 1.0 / N
        D = grid.divergence(N, h).toarray()
        G = grid.gradient(N, h).toarray()
        assert np.array_equal(D, -G.T)


@pytest.mark.parametrize("k,l", [(0, 1), (1, 0), (2, 3), (5, 7), (3, 3)])
def test_stokes_fourier_symbol(k, l):
    # For a single Fourier mode the MAC operators act by closed-form symbols:
    #   L: -(4/h^2)(sin^2(tx/2) + sin^2(ty/2)),  G^u: (1 - e^{-i tx})/h,
    #   -D: -((e^{i tx} - 1) u + (e^{i ty} - 1) v)/h.
    N, rho, dt, mu = 16, 1.3, 0.01, 0.07
    h = 1.0 / N
    K = grid.reduced_operator(N, h, rho, dt, mu, None)
    tx, ty = 2 * np.pi * k / N, 2 * np.pi * l / N
    j, i = np.divmod(np.arange(N * N), N)
    e = np.exp(1j * (tx * i + ty * j))
    uh, vh, ph = 0.3 - 0.2j, -0.5 + 0.1j, 0.7 + 0.4j
    x = np.concatenate([uh * e, vh * e, ph * e])
    y = K @ x.real + 1j * (K @ x.imag)
    lam = -(4 / h ** 2) * (np.sin(tx / 2) ** 2 + np.sin(ty / 2) ** 2)
    a0 = rho / dt - mu * lam
    ru = a0 * uh + (1 - np.exp(-1j * tx)) / h * ph
    rv = a0 * vh + (1 - np.exp(-1j * ty)) / h * ph
    rp = -((np.exp(1j * tx) - 1) * uh + (np.exp(1j * ty) - 1) * vh) / h
    want = np.concatenate([ru * e, rv * e, rp * e])
    assert np.allclose(y, want, rtol=0, atol=1e-10 * np.abs(want).max())


def _random_system(N=16, M=37, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (M, 2))
    return W.System(name="rand", N=N, L=1.0, rho=1.0, mu=0.01, dt=0.01, law=W.LAW_MEMBRANE,
                    closed=True, X=X, ds=0.02, omega=rng.uniform(0.01, 0.03, M), k_stretch=3.0)


def test_spread_interp_adjoint():
    # Sec. 2: <u, S F>_E = <J u, F>_L with <a,b>_E = h^2 sum a b, <A,B>_L = sum omega A.B
    s = _random_system()
    h = s.h
    S = ib.spreading_matrix(s.N, h, s.X, s.omega)
    J = ib.interpolation_matrix(s.N, h, s.X)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(2 * s.N ** 2)
    F = rng.standard_normal(2 * s.M)
    lhs = h ** 2 * u @ (S @ F)
    rhs = np.concatenate([s.omega, s.omega]) @ ((J @ u) * F)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_spread_is_scaled_transpose_for_uniform_weights():
    # App. A: with omega_k = ds, S = (ds / h^2) J^T entrywise
    s = W.membrane_ellipse(32, 1e4)
    S = ib.spreading_matrix(s.N, s.h, s.X, s.omega).toarray()
    J = ib.interpolation_matrix(s.N, s.h, s.X).toarray()
    assert np.allclose(S, (s.ds / s.h ** 2) * J.T, rtol=1e-15, atol=0)


def test_interpolation_reproduces_constant_and_linear_fields():
    # The kernel's zeroth and first moments make J exact on constants and on linear fields:
    # interpolating the faces' own x (or y) coordinate returns the marker's coordinate.
    N = 32
    h = 1.0 / N
    rng = np.random.default_rng(5)
    X = rng.uniform(0.3, 0.7, (50, 2))          # away from the periodic seam
    J = ib.interpolation_matrix(N, h, X)
    assert np.allclose(J @ np.ones(2 * N * N), 1.0, atol=1e-14)
    j, i = np.divmod(np.arange(N * N), N)
    xu, yu = i * h, (j + 0.5) * h                # u faces
    xv, yv = (i + 0.5) * h, j * h                # v faces
    M = X.shape[0]
    Ux = J @ np.concatenate([xu, xv])
    Uy = J @ np.concatenate([yu, yv])
    assert np.allclose(Ux[:M], X[:, 0], atol=1e-14) and np.allclose(Ux[M:], X[:, 0], atol=1e-14)
    assert np.allclose(Uy[:M], X[:, 1], atol=1e-14) and np.allclose(Uy[M:], X[:, 1], atol=1e-14)


def test_force_matrices_closed_form_spectra():
    M, ds = 40, 0.013
    m = np.arange(M)
    s2 = np.sin(np.pi * m / M) ** 2
    E = ib.force_matrix(W.LAW_MEMBRANE, M, ds, 0, 7.0, 0).toarray()[:M, :M]
    assert np.allclose(E, E.T)
    assert np.allclose(np.sort(np.linalg.eigvalsh(E)), np.sort(-(4 * 7.0 / ds ** 2) * s2),
                       rtol=1e-12, atol=1e-9 * 7.0 / ds ** 2)
    E = ib.force_matrix(W.LAW_BEAM, M, ds, 0, 2.0, 0.5).toarray()[:M, :M]
    want = -(4 * 2.0 / ds ** 2) * s2 - (16 * 0.5 / ds ** 4) * s2 ** 2
    assert np.allclose(np.sort(np.linalg.eigvalsh(E)), np.sort(want), rtol=1e-10,
                       atol=1e-9 * 16 * 0.5 / ds ** 4)
    E = ib.force_matrix(W.LAW_TARGET, M, ds, 3.5, 0, 0).toarray()
    assert np.array_equal(E, -3.5 * np.eye(2 * M))


@pytest.mark.parametrize("mk", [lambda: W.target_circle(16, 40, 1e3, 1e-3),
                                lambda: W.membrane_ellipse(16, 1e4),
                                lambda: W.beam_curve(16, 48, 1.0, 10.0)])
def test_eulerian_elasticity_triple_product_symmetry_sign(mk):
    s = mk()
    EE, pat = ib.eulerian_elasticity(s)
    S = ib.spreading_matrix(s.N, s.h, s.X, s.omega).toarray()
    J = ib.interpolation_matrix(s.N, s.h, s.X).toarray()
    E = ib.force_matrix(s.law, s.M, s.ds, s.k_target, s.k_stretch, s.k_bend).toarray()
    dense = S @ E @ J
    scale = np.abs(dense).max()
    assert np.allclose(EE.toarray(), dense, atol=1e-13 * scale, rtol=0)
    assert np.allclose(dense, dense.T, atol=1e-12 * scale)
    ev = np.linalg.eigvalsh(0.5 * (dense + dense.T))
    assert ev.max() <= 1e-10 * scale                 # E_E negative semidefinite (Sec. 1)
    A = grid.A0(s.N, s.h, s.rho, s.dt, s.mu).toarray() - s.dt * dense
    np.linalg.cholesky(0.5 * (A + A.T))             # A = A0 - dt E_E is SPD


def _brute_pattern(s):
    """(k,l) in the pattern iff some markers a, b with E_ab structurally nonzero have face k
    within kernel reach (< 2h per axis, periodic) of a and face l within reach of b."""
    N, h, M = s.N, s.h, s.M
    j, i = np.divmod(np.arange(N * N), N)
    pos = {0: (i * h, (j + 0.5) * h), 1: ((i + 0.5) * h, j * h)}
    reach = np.zeros((2, M, N * N), dtype=bool)
    for c in (0, 1):
        fx, fy = pos[c]
        for a in range(M):
            dx = (fx - s.X[a, 0] + 0.5) % 1.0 - 0.5
            dy = (fy - s.X[a, 1] + 0.5) % 1.0 - 0.5
            reach[c, a] = (np.abs(dx) < 2 * h) & (np.abs(dy) < 2 * h)
    bw = 0 if s.law == 0 else (2 if (s.law == 2 and s.k_bend) else 1)
    Eb = np.zeros((M, M), dtype=bool)
    for a in range(M):
        for d in range(-bw, bw + 1):
            Eb[a, (a + d) % M] = True
    out = np.zeros((2 * N * N, 2 * N * N), dtype=bool)
    for c in (0, 1):
        R = reach[c].astype(np.int64)                  # M x N^2
        blk = (R.T @ Eb.astype(np.int64) @ R) > 0
        out[c * N * N:(c + 1) * N * N, c * N * N:(c + 1) * N * N] = blk
    return out


@pytest.mark.parametrize("mk", [lambda: W.target_circle(16, 40, 1e3, 1e-3),
                                lambda: W.membrane_ellipse(16, 1e4),
                                lambda: W.beam_curve(16, 48, 1.0, 10.0),
                                lambda: W.paper_target_rows(16)])
def test_elasticity_pattern_brute_force(mk):
    s = mk()
    _, pat = ib.eulerian_elasticity(s)
    assert np.array_equal(pat.toarray(), _brute_pattern(s))
