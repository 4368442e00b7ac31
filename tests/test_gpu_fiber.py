"""GPU parity for the nonlinear fiber law (Sec. 5.3) on a periodic stand-in of the fiber
benchmark's domain: its Newton tangent couples u and v in E_E, which every layer (assembly,
Galerkin levels, CAV sets, local matrices, both smoothers) must carry.  Against the oracle,
through the C ABI, on the same seeded configuration:

  * E_E on every level: pattern bit-exact, values within 1e-13 of the largest (summation
    order), cross-component entries present;
  * CAV patch sets bit-exact on every level; the finest level's average and largest patch
    printed beside the paper's fiber table;
  * the right-hand side S F(X) of the first step within 1e-12;
  * one additive and one coloured sweep per level within 1e-11;
  * FGMRES to 1e-9 relative to ||r_0|| (the paper's fiber tolerance): counts within one of
    the oracle's for both smoothers.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import colouring as ocol, fgmres as ofg, ib as oib, multigrid as omg, smoother as osm
from tests.gpu_helpers import gpu_ee_csr, host, rel, torch_dev

pytestmark = pytest.mark.gpu

ALPHA = 0.85
# the paper's fiber table: average and largest CAV patch on the finest level
PAPER_PATCH = {16: (11.76, 201), 32: (7.85, 198)}


class Pair:
    pass


@pytest.fixture(scope="module", params=[16, 32])
def pair(request):
    from paper_2608_14310_b300 import api
    P = Pair()
    P.Np = request.param
    P.rec = W.fiber_periodic(request.param)
    P.levels = omg.build_hierarchy(P.rec, 8, "cav")
    P.sys = api.ib_setup(P.rec)
    P.h_add = api.cav_setup(P.sys, nu_pre=2, nu_post=2, alpha=ALPHA, precision="fp64")
    P.h_col = api.cav_setup(P.sys, nu_pre=1, nu_post=1, precision="fp64", smoother="coloured")
    return P


def test_fiber_ee_all_levels(pair):
    NN = pair.rec.N ** 2
    for l, lev in enumerate(pair.levels):
        G = gpu_ee_csr(pair.h_add, l)
        O = lev.EE.tocsr()
        O.sort_indices()
        assert np.array_equal(G.indptr, O.indptr) and np.array_equal(G.indices, O.indices), l
        scale = np.abs(O.data).max()
        assert np.abs(G.data - O.data).max() <= 1e-13 * scale, l
        if l == 0:
            NNl = lev.N ** 2
            assert np.abs(G[:NNl, NNl:]).max() > 1e-3 * scale
    assert pair.levels[0].N ** 2 == NN


def test_fiber_patch_sets(pair):
    from paper_2608_14310_b300 import api
    for l, lev in enumerate(pair.levels[:-1]):
        off, dofs = api.cav_patch_export(pair.h_add, l)
        want_off = np.concatenate([[0], np.cumsum([len(p) for p in lev.patches])])
        assert np.array_equal(off, want_off), l
        assert np.array_equal(dofs, np.concatenate(lev.patches).astype(np.int32)), l
    sz = np.diff(api.cav_patch_export(pair.h_add, 0)[0])
    avg, mx = PAPER_PATCH[pair.Np]
    print(f"fiber N={pair.Np}: finest-level patches avg {sz.mean():.2f} (paper {avg}), max {sz.max()} (paper {mx})")


def test_fiber_rhs(pair):
    from paper_2608_14310_b300 import api
    n = 3 * pair.rec.N ** 2
    b = torch_dev(np.zeros(n))
    api.ib_step_rhs(pair.sys, None, None, b)
    want = oib.first_step_rhs(pair.rec)
    assert np.abs(host(b) - want).max() <= 1e-12 * np.abs(want).max()


def test_fiber_sweeps(pair):
    from paper_2608_14310_b300 import api
    rng = np.random.default_rng(17)
    for l, lev in enumerate(pair.levels[:-1]):
        n = 3 * lev.N ** 2
        b = rng.uniform(-1, 1, n)
        b[2 * lev.N ** 2:] -= b[2 * lev.N ** 2:].mean()
        w0 = rng.uniform(-1, 1, n) * 1e-2
        w = torch_dev(w0)
        api.cav_sweep(pair.h_add, l, torch_dev(b), w)
        want = osm.additive_sweep(lev.KE, lev.solvers, lev.theta, w0, b, lev.N, ALPHA)
        assert rel(host(w), want) <= 1e-11, ("additive", l)
        w = torch_dev(w0)
        api.cav_sweep(pair.h_col, l, torch_dev(b), w)
        want = ocol.coloured_sweep(lev.KE, lev.solvers, omg.level_colours(lev), w0, b, lev.N)
        assert rel(host(w), want) <= 1e-11, ("coloured", l)


def test_fiber_fgmres(pair):
    from paper_2608_14310_b300 import api
    b = oib.first_step_rhs(pair.rec)
    K = pair.levels[0].KE
    for tag, h, nu, mode, a in (("additive", pair.h_add, 2, "additive", ALPHA),
                                ("coloured", pair.h_col, 1, "coloured", 1.0)):
        x = torch_dev(np.zeros(b.size))
        info = api.fgmres_solve(pair.sys, h, torch_dev(b), x, rtol=1e-9, maxit=150, rel_to=1)
        _, io = ofg.fgmres(lambda v: K @ v, b, lambda r: omg.vcycle(pair.levels, r, nu, nu, mode, a),
                           rtol=1e-9, maxit=150, ref="r0")
        assert info["converged"] == 1 and io["converged"], tag
        assert abs(info["iters"] - io["iters"]) <= 1, (tag, info["iters"], io["iters"])
        assert np.linalg.norm(b - K @ host(x)) <= 2e-9 * np.linalg.norm(b)
        print(f"fiber N={pair.Np} {tag}: gpu its {info['iters']} oracle its {io['iters']}")


def test_fiber_descriptor_refusals():
    from dataclasses import replace
    from paper_2608_14310_b300 import api
    rec = W.fiber_periodic(16)
    for bad in (replace(rec, closed=True), replace(rec, X=rec.X[:-1], omega=rec.omega[:-1]),
                replace(rec, k_target=1.0)):
        with pytest.raises(api.IBError) as e:
            api.ib_setup(bad)
        assert e.value.status == api.IB_ERR_INVALID
