"""The coarsest level's direct solve (Sec. 4) with a larger coarsest grid, factorised on every
SM: both grid-parallel Gauss-Jordan kernels (blocked in panels, the default where a panel fits
in shared memory; column by column, CAV_COARSEST_COLUMNS=1) must give the one-CTA kernel's
inverse bit for bit (CAV_COARSEST_ONE_CTA=1 keeps the one-CTA kernel; both are set-up test
hooks), compared through the coarsest solve and a whole V-cycle, on the periodic (bordered) and
the channel's (plain) coarsest system; the two grid kernels agree bit for bit on the 32 x 32
coarsest level (3073 unknowns), which solves as the oracle does.
"""
import os

import numpy as np
import pytest

import ib_workloads as W
from oracle import multigrid as omg
from tests.gpu_helpers import host, rel, torch_dev

pytestmark = pytest.mark.gpu


HOOKS = {"one_cta": "CAV_COARSEST_ONE_CTA", "columns": "CAV_COARSEST_COLUMNS"}


def _setup(api, s, form, **kw):
    if form in HOOKS:
        os.environ[HOOKS[form]] = "1"
    try:
        return api.cav_setup(s, **kw)
    finally:
        for v in HOOKS.values():
            os.environ.pop(v, None)


@pytest.mark.parametrize("form", ["panels", "columns"])
@pytest.mark.parametrize("name", ["membrane64", "channel16"])
def test_grid_factorisation_equals_one_cta(name, form):
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(64, 1e4) if name == "membrane64" else W.fiber_channel(16)
    s = api.ib_setup(rec)
    kw = dict(coarsest_N=16, nu_pre=1, nu_post=1, alpha=0.85, precision="fp64")
    hg = _setup(api, s, form, **kw)
    h1 = _setup(api, s, "one_cta", **kw)
    L = api.cav_num_levels(hg)
    Nc = api.cav_get_level_info(hg, L - 1)["N"]
    assert Nc == 16
    b = W.rhs(Nc, 3)
    z1, z2 = torch_dev(np.zeros(b.size)), torch_dev(np.zeros(b.size))
    api.cav_coarse_solve(hg, torch_dev(b), z1)
    api.cav_coarse_solve(h1, torch_dev(b), z2)
    assert np.array_equal(host(z1), host(z2)), name
    r = rec.rhs()
    v1, v2 = torch_dev(np.zeros(r.size)), torch_dev(np.zeros(r.size))
    api.vcycle_apply(hg, torch_dev(r), v1)
    api.vcycle_apply(h1, torch_dev(r), v2)
    assert np.array_equal(host(v1), host(v2)), name


def test_panel_and_column_kernels_agree_on_3073_unknowns():
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(64, 1e4)
    s = api.ib_setup(rec)
    kw = dict(coarsest_N=32, nu_pre=1, nu_post=1, alpha=0.85, precision="fp64")
    hp = _setup(api, s, "panels", **kw)
    hc = _setup(api, s, "columns", **kw)
    b = W.rhs(32, 11)
    z1, z2 = torch_dev(np.zeros(b.size)), torch_dev(np.zeros(b.size))
    api.cav_coarse_solve(hp, torch_dev(b), z1)
    api.cav_coarse_solve(hc, torch_dev(b), z2)
    assert np.array_equal(host(z1), host(z2))


def test_coarsest_32_against_oracle():
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(64, 1e4)
    levels = omg.build_hierarchy(rec, 32, "cav")
    assert levels[-1].N == 32
    s = api.ib_setup(rec)
    h = api.cav_setup(s, coarsest_N=32, nu_pre=1, nu_post=1, alpha=0.85, precision="fp64")
    b = W.rhs(32, 7)
    z = torch_dev(np.zeros(b.size))
    api.cav_coarse_solve(h, torch_dev(b), z)
    want = omg.coarse_solve(levels[-1], b)
    e = rel(host(z), want)
    print(f"coarsest 32 x 32 (3073 unknowns with the border): rel. diff to the oracle {e:.2e}")
    assert e <= 1e-11
    x = torch_dev(np.zeros(3 * 64 * 64))
    info = api.fgmres_solve(s, h, torch_dev(rec.rhs()), x, rtol=1e-10, maxit=100)
    assert info["converged"] == 1, info


@pytest.mark.parametrize("form,nu_pre,nu_post", [("coloured_finest", 1, 1), ("coloured_finest_post_only", 0, 1)])
def test_bench_solve_with_coarsest_32(form, nu_pre, nu_post):
    """The bench's solve (N = 256 membrane, FP32 inverses, coloured finest level 1+1 or 0+1,
    additive 4+4 below, 32 x 32 coarsest) reaches 1e-10 in the oracle's own iteration count for
    the same V-cycle (tests/golden/bench_oracle_iterations.json, written by the oracle alone),
    within one."""
    import json
    import os as _os
    from paper_2608_14310_b300 import api
    with open(_os.path.join(_os.path.dirname(__file__), "golden", "bench_oracle_iterations.json")) as f:
        golden = json.load(f)["coarsest_32"][form]["iters"]
    rec = W.config2(256, 1e4)
    s = api.ib_setup(rec)
    h = api.cav_setup(s, coarsest_N=32, nu_pre=nu_pre, nu_post=nu_post, alpha=0.85, precision="fp32",
                      smoother="coloured", coloured_levels=1, nu_additive=4)
    x = torch_dev(np.zeros(3 * 256 * 256))
    info = api.fgmres_solve(s, h, torch_dev(rec.rhs()), x, rtol=1e-10, maxit=150, loop="device")
    print(f"bench solve {nu_pre}+{nu_post}, 32 x 32 coarsest: {info['iters']} iterations (oracle {golden}), "
          f"true relres {info['relres_true']:.2e}")
    assert info["converged"] == 1 and info["relres_true"] <= 1e-10
    assert abs(info["iters"] - golden) <= 1
