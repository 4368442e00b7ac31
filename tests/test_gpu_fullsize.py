"""Parity at the full bench and stress sizes, in the launch configuration the bench uses:
the elliptic membrane at N=256 (4N markers, kappa_s=1e4), the membrane's stiffness sweep at
N=128 (kappa_s = 1e2 and 1e6) and the stretched beam at N=512 (2048 markers, kappa_b=1e3,
kappa_s=1e5).

E_E patterns and CAV patch sets are compared bit for bit on every level (the oracle builds
them in seconds without factorising).  The sweep is checked on sampled velocity unknowns the
oracle can compute one by one: r = b - K_E w in full, then only the patches holding each
sampled unknown are factorised.  Tolerance from the arithmetic: the two sides' FP64
inverses of an equilibrated patch matrix differ by up to about cond * eps, so the sampled
corrections must agree to max(1e-9, 100 * cond_max * eps) of the largest sampled correction,
cond_max the largest 2-norm condition number among the factorised patches (the stiff beam's
patches reach ~1e9-1e10; the membrane's stay near 1e4).
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import multigrid as omg, smoother as osm
from tests.gpu_helpers import gpu_ee_csr, host, torch_dev

pytestmark = pytest.mark.gpu

ALPHA = 0.85
CASES = {"membrane256": (lambda: W.config2(256, 1e4), "fp32"),
         "membrane128_k1e2": (lambda: W.config2(128, 1e2), "fp32"),
         "membrane128_k1e6": (lambda: W.config2(128, 1e6), "fp32"),
         "beam512": (lambda: W.config3(), "bf16")}


class Full:
    pass


@pytest.fixture(scope="module", params=sorted(CASES))
def full(request):
    from paper_2608_14310_b300 import api
    mk, prec = CASES[request.param]
    F = Full()
    F.name, F.rec, F.prec = request.param, mk(), prec
    F.levels = omg.build_hierarchy(F.rec, 8, "cav", factor=False)
    F.sys = api.ib_setup(F.rec)
    F.h = api.cav_setup(F.sys, nu_pre=2, nu_post=2, alpha=ALPHA, precision=prec)
    F.h64 = api.cav_setup(F.sys, nu_pre=2, nu_post=2, alpha=ALPHA, precision="fp64")
    return F


def test_full_patterns_and_patch_sets(full):
    from paper_2608_14310_b300 import api
    for l, lev in enumerate(full.levels):
        G = gpu_ee_csr(full.h, l)
        O = lev.EE.tocsr()
        O.sort_indices()
        assert np.array_equal(G.indptr, O.indptr) and np.array_equal(G.indices, O.indices), l
        assert np.abs(G.data - O.data).max() <= 1e-13 * np.abs(O.data).max(), l
        if l == len(full.levels) - 1:
            continue
        off, dofs = api.cav_patch_export(full.h, l)
        want_off = np.concatenate([[0], np.cumsum([len(p) for p in lev.patches])])
        assert np.array_equal(off, want_off), l
        assert np.array_equal(dofs, np.concatenate(lev.patches).astype(np.int32)), l


def test_full_sweep_sampled(full):
    from paper_2608_14310_b300 import api
    if full.name == "membrane256":
        pytest.skip("compared as whole vectors on every level in test_gpu_fullsize_sweep.py")
    lev = full.levels[0]
    N = lev.N
    NN = N * N
    rng = np.random.default_rng(31)
    n = 3 * NN
    b = rng.uniform(-1, 1, n)
    w0 = rng.uniform(-1, 1, n) * 1e-3
    w = torch_dev(w0)
    api.cav_sweep(full.h64, 0, torch_dev(b), w)
    got = host(w)
    r = b - lev.KE @ w0
    sizes = np.array([len(p) for p in lev.patches])
    owner = np.repeat(np.arange(len(lev.patches)), sizes)
    alld = np.concatenate(lev.patches)
    big_dofs = np.unique(np.concatenate([p for p in lev.patches if len(p) > 5]))
    vel_big = big_dofs[big_dofs < 2 * NN]
    samples = np.concatenate([rng.choice(vel_big, 10, replace=False), rng.integers(0, 2 * NN, 6)])
    cache = {}
    worst, scale = 0.0, 0.0
    for k in samples:
        ps = owner[alld == k]
        s = 0.0
        for p in ps:
            if p not in cache:
                cache[p] = osm.PatchSolver(lev.KE, lev.patches[p], NN, 2 * NN)
            sol = cache[p]
            s += sol.apply(r[sol.dofs])[np.searchsorted(sol.dofs, k)]
        corr = ALPHA * s / len(ps)
        worst = max(worst, abs((got[k] - w0[k]) - corr))
        scale = max(scale, abs(corr))
    # X is the inverse of the equilibrated patch matrix, so cond(X) is that matrix's condition number
    cond = max(np.linalg.cond(sol.X) for sol in cache.values())
    tol = max(1e-9, 100 * cond * np.finfo(float).eps)
    assert worst <= tol * scale, (worst, scale, cond)
    assert abs(got[2 * NN:].mean()) <= 1e-12 * max(1.0, np.abs(got[2 * NN:]).max())
    print(f"{full.name}: sampled sweep max abs diff {worst:.2e} of max correction {scale:.2e}, "
          f"cond_max {cond:.2e}")


def test_full_fgmres(full):
    from paper_2608_14310_b300 import api
    b = full.rec.rhs()
    K = full.levels[0].KE
    out = {}
    for tag, h in (("fp64", full.h64), (full.prec, full.h)):
        x = torch_dev(np.zeros(b.size))
        info = api.fgmres_solve(full.sys, h, torch_dev(b), x, rtol=1e-10, maxit=150)
        xg = host(x)
        out[tag] = (info, np.linalg.norm(b - K @ xg) / np.linalg.norm(b))
    print(full.name, {k: (v[0]["iters"], v[0]["converged"], f"{v[1]:.2e}") for k, v in out.items()})
    i64, r64 = out["fp64"]
    im, rm = out[full.prec]
    # the mixed form reaches the level the FP64 form reaches (1e-10 where that is attainable)
    assert rm <= max(2e-10, 10 * r64)
    if i64["converged"]:
        assert im["converged"] == 1
