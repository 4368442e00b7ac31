"""cav_refactor: a hierarchy rebuilt numerically for a new E_E on an unchanged pattern (the next
Newton iterate of a fiber time step, Sec. 5.3) equals a hierarchy set up from scratch for the
same system, bit for bit: E_E on every level, one sweep per level, the V-cycle and the FGMRES
solve.  When the pattern changes (the markers moved across faces) the call declines and
leaves the hierarchy as it was.
"""
from dataclasses import replace

import numpy as np
import pytest

import ib_workloads as W
from tests.gpu_helpers import gpu_ee_csr, host, torch_dev

pytestmark = pytest.mark.gpu


def _moved(rec, amount, seed):
    rng = np.random.default_rng(seed)
    return rec.X + amount * rec.ds * rng.uniform(-1, 1, rec.X.shape)


@pytest.mark.parametrize("bc,smoother,precision", [("channel", "coloured", "fp64"), ("channel", "additive", "fp32"),
                                                   ("periodic", "coloured", "fp32")])
def test_refactor_equals_fresh_setup(bc, smoother, precision):
    from paper_2608_14310_b300 import api
    rec = W.fiber_channel(16) if bc == "channel" else W.fiber_periodic(16)
    kw = dict(kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, alpha=0.85, smoother=smoother, precision=precision)
    sysm = api.ib_setup(rec)
    h = api.cav_setup(sysm, **kw)
    # the next Newton iterate: the force and tangent at a nearby configuration, S and J unchanged
    rec_b = replace(rec, meta={**rec.meta, "X_lin": _moved(rec, 0.2, 3)})
    api.ib_update_structure(sysm, rec_b)
    assert api.cav_refactor(h, sysm)
    fresh = api.cav_setup(sysm, **kw)
    L = api.cav_num_levels(h)
    for l in range(L):
        a, b = gpu_ee_csr(h, l), gpu_ee_csr(fresh, l)
        assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)
        assert np.array_equal(a.data, b.data), l
    rng = np.random.default_rng(7)
    for l in range(L - 1):
        N = api.cav_get_level_info(h, l)["N"]
        bb = rng.uniform(-1, 1, 3 * N * N)
        w0 = rng.uniform(-1, 1, 3 * N * N) * 1e-2
        w1, w2 = torch_dev(w0), torch_dev(w0)
        api.cav_sweep(h, l, torch_dev(bb), w1)
        api.cav_sweep(fresh, l, torch_dev(bb), w2)
        assert np.array_equal(host(w1), host(w2)), l
    b = rec.rhs()
    x1, x2 = torch_dev(np.zeros(b.size)), torch_dev(np.zeros(b.size))
    i1 = api.fgmres_solve(sysm, h, torch_dev(b), x1, rtol=1e-10, maxit=150)
    i2 = api.fgmres_solve(sysm, fresh, torch_dev(b), x2, rtol=1e-10, maxit=150)
    assert i1["converged"] == 1 and i1["iters"] == i2["iters"]
    assert np.array_equal(host(x1), host(x2))


def test_refactor_declines_a_changed_pattern():
    from paper_2608_14310_b300 import api
    rec = W.fiber_channel(16)
    sysm = api.ib_setup(rec)
    h = api.cav_setup(sysm, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, smoother="coloured", precision="fp64")
    b = rec.rhs()
    w0 = np.full(b.size, 1e-3)
    before = torch_dev(w0)
    api.cav_sweep(h, 0, torch_dev(b), before)
    # a new time step whose markers moved by two cells: S and J change, and with them E_E's pattern
    moved = replace(rec, X=rec.X + np.array([2.0 * rec.h, 0.0]))
    other = api.ib_setup(moved)
    assert not api.cav_refactor(h, other)
    after = torch_dev(w0)
    api.cav_sweep(h, 0, torch_dev(b), after)
    assert np.array_equal(host(before), host(after))
