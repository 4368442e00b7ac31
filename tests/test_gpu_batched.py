"""Batched solves of uneven systems (fgmres_solve_batched) and the patch-apply autotuner.

Every system in a batch runs the same kernels in the same order as when solved alone, only
on its own stream, so the batched results must equal the individual ones bit for bit; the
autotuner only chooses among kernel variants that accumulate identically, so autotuned
hierarchies must give the same bits too.  Both are checked against the oracle's iteration
counts as well.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import fgmres as ofg, multigrid as omg
from tests.gpu_helpers import host, torch_dev

pytestmark = pytest.mark.gpu

ALPHA = 0.85


def _systems():
    return [W.config1(),
            W.membrane_ellipse(32, 1e3),
            W.beam_curve(24, 96, k_bend=1e-2, k_stretch=1.0),
            W.target_circle(16, 48, 1e3, 1e-2),
            W.membrane_ellipse(16, 1e2)]


def test_batched_equals_individual_and_oracle():
    from paper_2608_14310_b300 import api
    recs = _systems()
    syss, hs, bs = [], [], []
    for rec in recs:
        s = api.ib_setup(rec)
        syss.append(s)
        hs.append(api.cav_setup(s, nu_pre=2, nu_post=2, alpha=ALPHA, precision="fp64"))
        bs.append(rec.rhs())
    single = []
    for s, h, b in zip(syss, hs, bs):
        x = torch_dev(np.zeros(b.size))
        info = api.fgmres_solve(s, h, torch_dev(b), x, rtol=1e-10, maxit=150)
        single.append((info, host(x)))
    xs = [torch_dev(np.zeros(b.size)) for b in bs]
    infos = api.fgmres_solve_batched(syss, hs, [torch_dev(b) for b in bs], xs, rtol=1e-10, maxit=150)
    for (i1, x1), i2, x2, rec, b in zip(single, infos, xs, recs, bs):
        assert i1["iters"] == i2["iters"] and i2["converged"] == 1
        assert np.array_equal(x1, host(x2)), rec.name
        levels = omg.build_hierarchy(rec, 8, "cav")
        K = levels[0].KE
        _, io = ofg.fgmres(lambda v: K @ v, b, lambda r: omg.vcycle(levels, r, 2, 2, "additive", ALPHA),
                           rtol=1e-10, maxit=150)
        assert abs(io["iters"] - i2["iters"]) <= 1, (rec.name, io["iters"], i2["iters"])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_autotune_is_result_neutral(precision):
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(64, 1e4)
    s = api.ib_setup(rec)
    h0 = api.cav_setup(s, nu_pre=2, nu_post=2, alpha=ALPHA, precision=precision)
    h1 = api.cav_setup(s, nu_pre=2, nu_post=2, alpha=ALPHA, precision=precision, autotune=True)
    for l in range(api.cav_num_levels(h1) - 1):
        info = api.cav_get_level_info(h1, l)
        if info["n_enlarged"]:
            assert any(t > 0 for t in info["apply_us"]), info
    b = rec.rhs()
    outs = []
    for h in (h0, h1):
        x = torch_dev(np.zeros(b.size))
        info = api.fgmres_solve(s, h, torch_dev(b), x, rtol=1e-10, maxit=150)
        outs.append((info["iters"], host(x)))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])
    lev0 = api.cav_get_level_info(h1, 0)
    print(precision, "variant times (us):", [round(t, 1) for t in lev0["apply_us"]], "chosen", lev0["apply_variant"])


@pytest.mark.parametrize("coloured_levels", [0, 1])
def test_batched_coloured_equals_individual(coloured_levels):
    # the coloured smoother (every level, or the finest only with the additive sweep below):
    # its class steps launch with programmatic dependent launch inside each system's V-cycle
    # graph, on the system's own stream; batching must not change a bit
    from paper_2608_14310_b300 import api
    recs = _systems()
    syss, hs, bs = [], [], []
    for rec in recs:
        s = api.ib_setup(rec)
        syss.append(s)
        hs.append(api.cav_setup(s, nu_pre=1, nu_post=1, alpha=ALPHA, precision="fp32", smoother="coloured",
                                coloured_levels=coloured_levels, nu_additive=2))
        bs.append(rec.rhs())
    single = []
    for s, h, b in zip(syss, hs, bs):
        x = torch_dev(np.zeros(b.size))
        info = api.fgmres_solve(s, h, torch_dev(b), x, rtol=1e-10, maxit=150)
        single.append((info, host(x)))
    xs = [torch_dev(np.zeros(b.size)) for b in bs]
    infos = api.fgmres_solve_batched(syss, hs, [torch_dev(b) for b in bs], xs, rtol=1e-10, maxit=150)
    for (i1, x1), i2, x2, rec in zip(single, infos, xs, recs):
        assert i1["iters"] == i2["iters"] and i2["converged"] == 1, rec.name
        assert np.array_equal(x1, host(x2)), rec.name
