"""GPU parity of the box smoother B(4,2) with restricted injection (Sec. 3.1, 3.3), the paper's
geometric comparator, against the oracle through the C ABI, on the same seeded inputs:

  * patch sets: bit-exact with the oracle's B(4,2) family on every smoothing level (blocks in
    lexicographic order of their lower-left cells);
  * colour classes over the blocks: bit-exact with the oracle's first-fit colouring;
  * one sweep per level: the class-by-class multiplicative sweep with restricted injection,
    ||w_gpu - w_oracle|| / ||w_oracle|| <= 1e-11 (the two sides' inverses of the 208 x 208
    equilibrated patch matrices differ by about cond * eps);
  * one V-cycle within 1e-10; FGMRES iteration counts within one of the oracle's;
  * the paper's target-point experiment (Sec. 5.2): counts within three of the printed
    B(4,2) counts at N = 32 and 64 (N = 128 printed); its beam counts are printed beside the
    paper's (a recorded deviation);
  * invalid descriptors are refused at set-up.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import fgmres as ofg, ib as oib, multigrid as omg
from tests.gpu_helpers import gpu_hierarchy, host, rel, torch_dev

pytestmark = pytest.mark.gpu

CASES = {
    "membrane32": lambda: W.membrane_ellipse(32, 1e4),
    "beam32": lambda: W.beam_curve(32, 96, 1.0, 10.0),
    "target_rows32": lambda: W.paper_target_rows(32),
}


class Pair:
    pass


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    rec = CASES[request.param]()
    P = Pair()
    P.name, P.rec = request.param, rec
    P.levels = omg.build_hierarchy(rec, 8, "box")
    P.sys, P.h = gpu_hierarchy(rec, kind="box", coarsest_N=8, nu_pre=1, nu_post=1, precision="fp64",
                               smoother="coloured")
    return P


def test_box_patch_sets_bit_exact(pair):
    from paper_2608_14310_b300 import api
    for l, lev in enumerate(pair.levels[:-1]):
        off, dofs = api.cav_patch_export(pair.h, l)
        assert off.size - 1 == (lev.N // 4) ** 2 == len(lev.patches)
        want_off = np.concatenate([[0], np.cumsum([len(p) for p in lev.patches])])
        assert np.array_equal(off, want_off), l
        assert np.array_equal(dofs, np.concatenate(lev.patches).astype(np.int32)), l
        info = api.cav_get_level_info(pair.h, l)
        assert info["n_patches"] == info["n_enlarged"] == len(lev.patches)
        assert info["max_n"] == 208


def test_box_classes_bit_exact(pair):
    from paper_2608_14310_b300 import api
    for l, lev in enumerate(pair.levels[:-1]):
        want = omg.level_colours(lev)
        got = api.cav_colour_export(pair.h, l)
        assert np.array_equal(got, want), l


def test_one_box_sweep_per_level(pair):
    from paper_2608_14310_b300 import api
    from oracle import colouring as ocol
    rng = np.random.default_rng(41)
    for l, lev in enumerate(pair.levels[:-1]):
        n = 3 * lev.N ** 2
        b = rng.uniform(-1, 1, n)
        b[2 * lev.N ** 2:] -= b[2 * lev.N ** 2:].mean()
        w0 = rng.uniform(-1, 1, n) * 1e-2
        w = torch_dev(w0)
        api.cav_sweep(pair.h, l, torch_dev(b), w)
        want = ocol.coloured_sweep(lev.KE, lev.solvers, omg.level_colours(lev), w0, b, lev.N, lev.inject)
        e = rel(host(w), want)
        assert e <= 1e-11, (l, e)


def test_box_vcycle_and_fgmres(pair):
    from paper_2608_14310_b300 import api
    b = pair.rec.rhs()
    z = torch_dev(np.zeros(b.size))
    api.vcycle_apply(pair.h, torch_dev(b), z)
    assert rel(host(z), omg.vcycle(pair.levels, b, 1, 1, "coloured")) <= 1e-10
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(pair.sys, pair.h, torch_dev(b), x, rtol=1e-10, maxit=150)
    K = pair.levels[0].KE
    _, io = ofg.fgmres(lambda v: K @ v, b, lambda r: omg.vcycle(pair.levels, r, 1, 1, "coloured"),
                       rtol=1e-10, maxit=150)
    assert info["converged"] == 1 and io["converged"]
    assert abs(info["iters"] - io["iters"]) <= 1, (info["iters"], io["iters"])
    assert np.linalg.norm(b - K @ host(x)) <= 2e-10 * np.linalg.norm(b)
    print(f"{pair.name}: box gpu its {info['iters']} oracle its {io['iters']}")


def _paper_solve(s, kind):
    from paper_2608_14310_b300 import api
    sys_, h = gpu_hierarchy(s, kind=kind, coarsest_N=8, nu_pre=1, nu_post=1, precision="fp64",
                            smoother="coloured")
    b = torch_dev(np.zeros(3 * s.N * s.N))
    api.ib_step_rhs(sys_, None, None, b)
    x = torch_dev(np.zeros(3 * s.N * s.N))
    return api.fgmres_solve(sys_, h, b, x, rtol=1e-10, maxit=150, rel_to=1)


# Sec. 5.2: B(4,2) counts printed for the target-point rows (8, 10, 11) and the beam (6, 13, 26)
@pytest.mark.parametrize("N,paper", [(32, 8), (64, 10), (128, 11)])
def test_paper_target_box_counts(N, paper):
    s = W.paper_target_rows(N)
    info = _paper_solve(s, "box")
    cav = _paper_solve(s, "cav")
    print(f"target N={N}: box {info['iters']} (paper {paper}), cav {cav['iters']}")
    assert info["converged"] == 1 and cav["converged"] == 1
    if N <= 64:  # the oracle's class-order counts (8 and 8) are within three of the paper's
        assert abs(info["iters"] - paper) <= 3, info
    if N == 32:
        levels = omg.build_hierarchy(s, 8, "box")
        K = levels[0].KE
        _, io = ofg.fgmres(lambda v: K @ v, oib.first_step_rhs(s),
                           lambda r: omg.vcycle(levels, r, 1, 1, "coloured"), rtol=1e-10, maxit=150, ref="r0")
        assert abs(info["iters"] - io["iters"]) <= 1, (info["iters"], io["iters"])


@pytest.mark.parametrize("N,paper", [(32, 6), (64, 13), (128, 26)])
def test_paper_beam_box_counts_recorded(N, paper):
    # the printed counts are not reproduced (this B(4,2) with restricted injection takes 20
    # iterations at N = 32 in the oracle too); both the growth under refinement and CAV's
    # flat counts are: box counts rise with N while CAV's stay near ten
    s = W.paper_beam(N)
    info = _paper_solve(s, "box")
    cav = _paper_solve(s, "cav")
    print(f"beam N={N}: box {info['iters']} conv {info['converged']} (paper {paper}), cav {cav['iters']}")
    assert cav["converged"] == 1
    assert info["iters"] > cav["iters"] or not info["converged"]


def test_box_descriptor_refusals():
    from paper_2608_14310_b300 import api
    sys_ = api.ib_setup(W.membrane_ellipse(32, 1e4))
    bad = [dict(kind="box", smoother="additive"),
           dict(kind="box", smoother="coloured", coloured_levels=1),
           dict(kind="box", smoother="coloured", precision="bf16"),
           dict(kind="box", smoother="coloured", box=(3, 1)),   # 32 is not a multiple of 3
           dict(kind="box", smoother="coloured", box=(4, 6)),   # b + 2 o >= 16 on the N = 16 level
           dict(kind="box", smoother="coloured", box=(0, 2))]
    for kw in bad:
        with pytest.raises(api.IBError) as e:
            api.cav_setup(sys_, **kw)
        assert e.value.status == api.IB_ERR_INVALID, kw


def test_box_fp32_inverses_reach_tolerance():
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(32, 1e4)
    sys_, h = gpu_hierarchy(rec, kind="box", coarsest_N=8, nu_pre=1, nu_post=1, precision="fp32",
                            smoother="coloured")
    b = rec.rhs()
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(sys_, h, torch_dev(b), x, rtol=1e-10, maxit=150)
    assert info["converged"] == 1 and info["relres_true"] <= 2e-10, info
    print(f"membrane32 box fp32: {info['iters']} its")
