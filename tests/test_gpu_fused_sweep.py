"""The additive sweep as one fused cooperative kernel (residual, patch apply, scatter and mean
removal between grid-wide barriers) against the same sweep as separate kernels.

Each part of the fused kernel is the separate kernel's block-level work, done in the same
order, so the two forms must agree bit for bit: one sweep per level (the cav_sweep form, with
the mean removal), a V-cycle (whose first sweep on each level starts from w = 0, skipping the
residual), an FGMRES solve, and the allocation-free sweep.  CAV_SWEEP_FORM (a set-up test hook)
forces one form.  Also checked: the autotuner times both forms and keeps the faster, and the
device-driven batched loop runs several fused hierarchies side by side.
"""
import os

import numpy as np
import pytest

import ib_workloads as W
from tests.gpu_helpers import host, torch_dev

pytestmark = pytest.mark.gpu

ALPHA = 0.85


def _setup(api, s, form, **kw):
    os.environ["CAV_SWEEP_FORM"] = form
    try:
        return api.cav_setup(s, **kw)
    finally:
        os.environ.pop("CAV_SWEEP_FORM", None)


CASES = {
    "membrane64-fp64": (lambda: W.membrane_ellipse(64, 1e4), "fp64"),
    "membrane64-fp32": (lambda: W.membrane_ellipse(64, 1e4), "fp32"),
    "membrane64-bf16": (lambda: W.membrane_ellipse(64, 1e4), "bf16"),
    "membrane256-fp32": (lambda: W.config2(256, 1e4), "fp32"),
    "channel32-fp64": (lambda: W.fiber_channel(32), "fp64"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fused_sweep_equals_separate_kernels(name):
    from paper_2608_14310_b300 import api
    make, precision = CASES[name]
    rec = make()
    s = api.ib_setup(rec)
    kw = dict(nu_pre=2, nu_post=2, alpha=ALPHA, precision=precision)
    hf = _setup(api, s, "fused", **kw)
    hs = _setup(api, s, "separate", **kw)
    L = api.cav_num_levels(hf)
    fused_levels = 0
    rng = np.random.default_rng(21)
    for l in range(L - 1):
        inf_f, inf_s = api.cav_get_level_info(hf, l), api.cav_get_level_info(hs, l)
        assert inf_s["sweep_form"] == 0
        if inf_f["n_enlarged"] > 0:
            assert inf_f["sweep_form"] == 1, (name, l)
            fused_levels += 1
        N = inf_f["N"]
        b = rng.uniform(-1, 1, 3 * N * N)
        w0 = 1e-2 * rng.uniform(-1, 1, 3 * N * N)
        w1, w2, w3 = torch_dev(w0), torch_dev(w0), torch_dev(w0)
        for _ in range(2):  # two sweeps in a row: the barrier state carries over launches
            api.cav_sweep(hf, l, torch_dev(b), w1)
            api.cav_sweep(hs, l, torch_dev(b), w2)
        assert np.array_equal(host(w1), host(w2)), (name, l)
        api.cav_sweep_noalloc(hf, l, torch_dev(b), w3)
        api.cav_sweep_noalloc(hf, l, torch_dev(b), w3)
        assert np.array_equal(host(w3), host(w2)), (name, l, "noalloc")
    assert fused_levels >= 1
    b = rec.rhs()
    z1, z2 = torch_dev(np.zeros(b.size)), torch_dev(np.zeros(b.size))
    api.vcycle_apply(hf, torch_dev(b), z1)
    api.vcycle_apply(hs, torch_dev(b), z2)
    assert np.array_equal(host(z1), host(z2)), name
    x1, x2 = torch_dev(np.zeros(b.size)), torch_dev(np.zeros(b.size))
    i1 = api.fgmres_solve(s, hf, torch_dev(b), x1, rtol=1e-10, maxit=150)
    i2 = api.fgmres_solve(s, hs, torch_dev(b), x2, rtol=1e-10, maxit=150)
    assert i1["iters"] == i2["iters"] and np.array_equal(host(x1), host(x2)), name
    assert i1["converged"] == 1 or precision == "bf16"


def test_autotuner_times_both_forms():
    from paper_2608_14310_b300 import api
    rec = W.config2(256, 1e4)
    s = api.ib_setup(rec)
    h = api.cav_setup(s, nu_pre=2, nu_post=2, alpha=ALPHA, precision="fp32", autotune=True)
    info = api.cav_get_level_info(h, 0)
    sep, fus = info["sweep_us"]
    print(f"finest-level sweep: separate kernels {sep:.1f} us, fused {fus:.1f} us, form {info['sweep_form']}")
    assert sep > 0 and fus > 0
    assert info["sweep_form"] == (1 if fus < sep else 0)


def test_fused_hierarchies_in_one_batched_graph():
    from paper_2608_14310_b300 import api
    recs = [W.membrane_ellipse(64, 1e4), W.beam_curve(96, 384, k_bend=1e-2, k_stretch=1.0),
            W.membrane_ellipse(128, 1e3), W.target_circle(64, 256, 1e3, 1e-2)]
    syss = [api.ib_setup(r) for r in recs]
    hs = [_setup(api, s, "fused", nu_pre=2, nu_post=2, alpha=ALPHA, precision="fp32") for s in syss]
    bs = [torch_dev(r.rhs()) for r in recs]
    single = []
    for s, h, b in zip(syss, hs, bs):
        x = torch_dev(np.zeros(b.numel()))
        single.append((api.fgmres_solve(s, h, b, x, rtol=1e-10, maxit=100), host(x)))
    xs = [torch_dev(np.zeros(b.numel())) for b in bs]
    infos = api.fgmres_solve_batched(syss, hs, bs, xs, rtol=1e-10, maxit=100, loop="device")
    for (i1, x1), i2, x2, r in zip(single, infos, xs, recs):
        assert i1["iters"] == i2["iters"], r.name
        assert np.array_equal(x1, host(x2)), r.name
