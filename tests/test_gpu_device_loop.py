"""The device-driven FGMRES loop (fgmres_desc.loop = 1): a solve, or a batch of solves, as one
CUDA graph launch whose iterations run under a conditional while node.

Every iteration launches the same kernels with the same arguments as the host-driven loop;
only the iteration index comes from device memory.  So the two loops must agree bit for bit
-- iterate, iteration count, residual history -- on every smoother and boundary condition,
in a batch of uneven systems as well, and through the cached graph's rebuilds (new vectors,
a refactored hierarchy, an updated system).
"""
from dataclasses import replace

import numpy as np
import pytest

import ib_workloads as W
from tests.gpu_helpers import host, torch_dev

pytestmark = pytest.mark.gpu

ALPHA = 0.85


def _pair(api, s, h, b, rtol=1e-10, maxit=150, rel_to=0, x0=None):
    out = []
    for loop in ("host", "device"):
        x = torch_dev(np.zeros(b.size) if x0 is None else x0.copy())
        info = api.fgmres_solve(s, h, torch_dev(b), x, rtol=rtol, maxit=maxit, rel_to=rel_to, loop=loop)
        out.append((info, host(x)))
    return out


def _same(a, b, what):
    (i1, x1), (i2, x2) = a, b
    assert i1["iters"] == i2["iters"], (what, i1["iters"], i2["iters"])
    assert i1["converged"] == i2["converged"], what
    assert np.array_equal(i1["history"], i2["history"]), what
    assert i1["relres_true"] == i2["relres_true"], what
    assert np.array_equal(x1, x2), what


@pytest.mark.parametrize("smoother,precision", [("additive", "fp64"), ("additive", "fp32"),
                                                ("coloured", "fp64"), ("coloured", "fp32")])
def test_device_loop_equals_host_loop(smoother, precision):
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(64, 1e4)
    s = api.ib_setup(rec)
    kw = dict(nu_pre=1, nu_post=1, coloured_levels=1, nu_additive=2) if smoother == "coloured" else \
        dict(nu_pre=2, nu_post=2)
    h = api.cav_setup(s, alpha=ALPHA, precision=precision, smoother=smoother, **kw)
    a, b = _pair(api, s, h, rec.rhs())
    assert a[0]["converged"] == 1
    _same(a, b, (smoother, precision))


def test_device_loop_on_the_channel():
    from paper_2608_14310_b300 import api
    rec = W.fiber_channel(16)
    s = api.ib_setup(rec)
    h = api.cav_setup(s, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, smoother="coloured", precision="fp64")
    a, b = _pair(api, s, h, rec.rhs(), rel_to=1)
    assert a[0]["converged"] == 1
    _same(a, b, "channel")


def test_device_loop_edge_cases():
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(32, 1e3)
    s = api.ib_setup(rec)
    h = api.cav_setup(s, nu_pre=2, nu_post=2, alpha=ALPHA, precision="fp64")
    b = rec.rhs()
    # b = 0: converged before the first iteration, x untouched
    a, d = _pair(api, s, h, np.zeros_like(b))
    assert d[0]["iters"] == 0 and d[0]["converged"] == 1 and not np.any(d[1])
    _same(a, d, "zero rhs")
    # maxit reached above tolerance
    a, d = _pair(api, s, h, b, rtol=1e-30, maxit=3)
    assert d[0]["iters"] == 3 and d[0]["converged"] == 0
    _same(a, d, "maxit")
    # a nonzero initial guess, residual relative to r0
    x0 = np.random.default_rng(3).uniform(-1, 1, b.size)
    a, d = _pair(api, s, h, b, rel_to=1, x0=x0)
    _same(a, d, "x0")
    # host buffers are refused with the device-driven loop
    with pytest.raises(api.IBError):
        api.fgmres_solve(s, h, b.copy(), np.zeros_like(b), loop="device")


def test_cached_graph_is_rebuilt_when_its_inputs_change():
    import torch
    from paper_2608_14310_b300 import api
    rec = W.fiber_channel(16)
    s = api.ib_setup(rec)
    h = api.cav_setup(s, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, smoother="coloured", precision="fp64")
    b = rec.rhs()
    bd = torch_dev(b)
    x = torch_dev(np.zeros(b.size))
    i1 = api.fgmres_solve(s, h, bd, x, rel_to=1, maxit=150, loop="device")
    x1 = host(x)
    # the same call again replays the cached graph
    c0 = api.ib_launch_count()
    x.zero_()
    i2 = api.fgmres_solve(s, h, bd, x, rel_to=1, maxit=150, loop="device")
    assert i2["iters"] == i1["iters"] and np.array_equal(host(x), x1)
    assert api.ib_launch_count() - c0 >= 12 * i2["iters"]  # the graph's kernels are counted
    # other vectors
    b2 = 0.5 * b
    x2 = torch.zeros_like(x)
    i3 = api.fgmres_solve(s, h, torch_dev(b2), x2, rel_to=1, maxit=150, loop="device")
    ref = api.fgmres_solve(s, h, torch_dev(b2), torch.zeros_like(x), rel_to=1, maxit=150)
    assert i3["iters"] == ref["iters"] and np.array_equal(i3["history"], ref["history"])
    # the next Newton iterate (force and tangent at a nearby configuration, E_E's pattern
    # unchanged): ib_update_structure, then cav_refactor
    X_lin = rec.X + 0.2 * rec.ds * np.random.default_rng(3).uniform(-1, 1, rec.X.shape)
    api.ib_update_structure(s, replace(rec, meta={**rec.meta, "X_lin": X_lin}))
    a, d = _pair(api, s, h, b, rel_to=1)   # the updated system with the old hierarchy
    _same(a, d, "updated system")
    assert api.cav_refactor(h, s)
    a, d = _pair(api, s, h, b, rel_to=1)
    _same(a, d, "refactored")


def test_batched_device_loop_equals_individual_solves():
    from paper_2608_14310_b300 import api
    recs = [W.config1(), W.membrane_ellipse(32, 1e3), W.beam_curve(24, 96, k_bend=1e-2, k_stretch=1.0),
            W.target_circle(16, 48, 1e3, 1e-2), W.membrane_ellipse(64, 1e6), W.membrane_ellipse(16, 1e2)]
    syss, hs, bs = [], [], []
    for rec in recs:
        s = api.ib_setup(rec)
        syss.append(s)
        hs.append(api.cav_setup(s, nu_pre=2, nu_post=2, alpha=ALPHA, precision="fp32"))
        bs.append(rec.rhs())
    single = []
    for s, h, b in zip(syss, hs, bs):
        x = torch_dev(np.zeros(b.size))
        info = api.fgmres_solve(s, h, torch_dev(b), x, rtol=1e-10, maxit=60)
        single.append((info, host(x)))
    bd = [torch_dev(b) for b in bs]
    xs = [torch_dev(np.zeros(b.size)) for b in bs]
    for rep in range(2):  # the second call replays the cached batch graph
        for x in xs:
            x.zero_()
        infos = api.fgmres_solve_batched(syss, hs, bd, xs, rtol=1e-10, maxit=60, loop="device")
        for (i1, x1), i2, x2, rec in zip(single, infos, xs, recs):
            assert i1["iters"] == i2["iters"] and i1["converged"] == i2["converged"], (rec.name, rep)
            assert i1["relres_true"] == i2["relres_true"], rec.name
            assert np.array_equal(x1, host(x2)), (rec.name, rep)
