"""Pins of the weighted additive sweep (Eq. additive_cav_saddle) with many overlapping
patches, the form the GPU's additive path is compared against:

    r = b - K_E w;  w <- w + alpha sum_i R_i^T Theta_i K_{E,i}^{-1} R_i r;  remove mean pressure,
    Theta_i = 1 / (number of patches holding each unknown).

Each pin is a result the mathematics fixes independently of the oracle's code:

  * repeated whole domain: the bordered whole-domain patch listed m times (Theta = 1/m); one
    sweep with alpha = 1 is an exact solve, whatever m;
  * diagonal operator, random overlapping cover: every patch's local solve returns r_k / d_k at
    each of its unknowns, so the Theta-weighted sum is r_k / d_k whatever the multiplicities,
    and one sweep gives w + alpha (b / d - w) with the mean pressure removed;
  * block-diagonal operator, one patch per block (no coupling between patches): one sweep from
    zero is block Jacobi, i.e. the direct solve of each block (mean pressure removed);
  * linearity in alpha: w_alpha - remove_mean(w) is alpha times the same correction on a CAV
    level of the membrane.

`test_planted_mistakes_fail_a_pin` plants plausible mistakes in copies of the sweep (Theta
dropped, squared or replaced by the count; alpha dropped or squared; the corrections of
overlapping patches overwritten instead of summed; the mean left in) and checks that each
fails at least one pin, while the oracle passes all of them.  Applying alpha before or after
the Theta-weighted sum is the same linear map and is not a mistake.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import ib_workloads as W
from oracle import grid, ib, multigrid, smoother

TOL = 1e-12


def _remove_mean(w, N):
    # written out here, independently of the oracle: the pressure block is the last N^2 entries
    out = np.array(w, dtype=np.float64, copy=True)
    out[2 * N * N:] -= np.sum(out[2 * N * N:]) / (N * N)
    return out


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------------------- the pins

def pin_repeated_whole_domain(sweep):
    """Worst relative residual after one sweep with the whole-domain patch listed m times."""
    s = W.target_circle(8, 24, 1e3, 1e-2)
    EE, _ = ib.eulerian_elasticity(s)
    N = 8
    K = grid.reduced_operator(N, s.h, s.rho, s.dt, s.mu, EE)
    n = K.shape[0]
    b = s.rhs()
    worst = 0.0
    for m in (1, 2, 3):
        solvers = [smoother.PatchSolver(K, np.arange(n), N * N, 2 * N * N) for _ in range(m)]
        theta = smoother.partition_weights([sv.dofs for sv in solvers], n)
        assert np.all(theta == 1.0 / m)
        w = sweep(K, solvers, theta, np.zeros(n), b, N, 1.0)
        worst = max(worst, np.linalg.norm(b - K @ w) / np.linalg.norm(b))
    return worst


def _random_cover(n, rng, max_mult=4, size=(3, 9)):
    """Patches (sorted index arrays) covering every one of n unknowns 1..max_mult times."""
    need = rng.integers(1, max_mult + 1, n)
    have = np.zeros(n, dtype=int)
    patches = []
    while np.any(have < need):
        short = np.nonzero(have < need)[0]
        k = int(rng.integers(*size))
        p = set(rng.choice(short, min(k, short.size), replace=False).tolist())
        p |= set(rng.choice(n, 2, replace=False).tolist())  # overlap with arbitrary unknowns
        p = np.array(sorted(p))
        patches.append(p)
        have[p] += 1
    return patches


def pin_diagonal_overlapping(sweep):
    """Worst relative error against the closed form on a diagonal operator."""
    rng = np.random.default_rng(20261203)
    N = 4
    n = 3 * N * N
    worst = 0.0
    for alpha in (1.0, 0.85):
        d = rng.uniform(0.5, 3.0, n) * rng.choice([-1.0, 1.0], n)
        K = sp.diags(d).tocsr()
        patches = _random_cover(n, rng)
        counts = np.zeros(n)
        for p in patches:
            counts[p] += 1
        assert counts.max() >= 3 and counts.min() >= 1
        solvers = [smoother.PatchSolver(K, p) for p in patches]
        theta = smoother.partition_weights(patches, n)
        b = rng.uniform(-1, 1, n)
        w0 = rng.uniform(-1, 1, n)
        want = _remove_mean(w0 + alpha * (b / d - w0), N)
        got = sweep(K, solvers, theta, w0, b, N, alpha)
        worst = max(worst, _rel(got, want))
    return worst


def pin_block_jacobi(sweep):
    """Worst relative error against the direct solve of a block-diagonal operator."""
    rng = np.random.default_rng(77)
    N = 4
    n = 3 * N * N
    perm = rng.permutation(n)
    cuts = np.sort(rng.choice(np.arange(1, n), 9, replace=False))
    blocks = [np.sort(x) for x in np.split(perm, cuts)]
    A = np.zeros((n, n))
    for blk in blocks:
        m = blk.size
        B = rng.standard_normal((m, m))
        B += np.diag(np.sign(np.diag(B)) * (np.abs(B).sum(1) + 1.0))  # non-singular
        A[np.ix_(blk, blk)] = B
    K = sp.csr_matrix(A)
    solvers = [smoother.PatchSolver(K, blk) for blk in blocks]
    theta = smoother.partition_weights(blocks, n)
    b = rng.uniform(-1, 1, n)
    want = _remove_mean(np.linalg.solve(A, b), N)
    got = sweep(K, solvers, theta, np.zeros(n), b, N, 1.0)
    return _rel(got, want)


_MEMBRANE = {}


def _membrane_level():
    if "lev" not in _MEMBRANE:
        _MEMBRANE["lev"] = multigrid.build_hierarchy(W.membrane_ellipse(16, 1e4), 8, "cav")[0]
    return _MEMBRANE["lev"]


def pin_alpha_linearity(sweep):
    """Relative deviation of the alpha = 0.5 correction from half the alpha = 1 correction."""
    lev = _membrane_level()
    N = lev.N
    n = 3 * N * N
    rng = np.random.default_rng(5)
    b = rng.uniform(-1, 1, n)
    w0 = rng.uniform(-1, 1, n) * 1e-2
    base = _remove_mean(w0, N)
    c1 = sweep(lev.KE, lev.solvers, lev.theta, w0, b, N, 1.0) - base
    c2 = sweep(lev.KE, lev.solvers, lev.theta, w0, b, N, 0.5) - base
    c3 = sweep(lev.KE, lev.solvers, lev.theta, w0, b, N, 0.25) - base
    return max(_rel(2.0 * c2, c1), _rel(4.0 * c3, c1))


PINS = [pin_repeated_whole_domain, pin_diagonal_overlapping, pin_block_jacobi, pin_alpha_linearity]


# ------------------------------------------------------------------- oracle passes them

@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_oracle_additive_sweep_meets_pin(pin):
    assert pin(smoother.additive_sweep) <= TOL


def test_membrane_level_has_real_overlap():
    # the linearity pin runs on a level whose patches overlap with multiplicities above 2
    lev = _membrane_level()
    assert np.max(1.0 / lev.theta) >= 3
    assert sum(len(s.dofs) > 5 for s in lev.solvers) > 0


# ------------------------------------------------------------------- planted mistakes

def _mutant(kind):
    def sweep(KE, solvers, theta, w, b, N, alpha=1.0):
        r = b - KE @ w
        corr = np.zeros_like(w)
        for s in solvers:
            d = s.apply(r[s.dofs])
            if kind == "theta_dropped":
                corr[s.dofs] += d
            elif kind == "theta_squared":
                corr[s.dofs] += theta[s.dofs] ** 2 * d
            elif kind == "theta_is_count":
                corr[s.dofs] += d / theta[s.dofs]
            elif kind == "overwrite":
                corr[s.dofs] = theta[s.dofs] * d
            else:
                corr[s.dofs] += theta[s.dofs] * d
        if kind == "alpha_dropped":
            out = w + corr
        elif kind == "alpha_squared":
            out = w + alpha * alpha * corr
        else:
            out = w + alpha * corr
        if kind == "mean_kept":
            return out
        return smoother.remove_mean_pressure(out, N)
    sweep.__name__ = kind
    return sweep


MUTANTS = ["theta_dropped", "theta_squared", "theta_is_count", "overwrite", "alpha_dropped",
           "alpha_squared", "mean_kept"]


@pytest.mark.parametrize("kind", MUTANTS)
def test_planted_mistakes_fail_a_pin(kind):
    bad = _mutant(kind)
    errs = {p.__name__: p(bad) for p in PINS}
    assert max(errs.values()) > 1e3 * TOL, errs


def test_unmutated_copy_passes():
    # the mutant scaffold itself, with no mistake planted, meets every pin
    ok = _mutant("none")
    assert max(p(ok) for p in PINS) <= TOL
