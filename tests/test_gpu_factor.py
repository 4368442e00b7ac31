"""The batched FP64 patch factorisation (Sec. 3.3): the shared-memory kernel on CTA pairs gives
the same inverses, bit for bit, as the one-CTA global-memory kernel (CAV_FACTOR_GLOBAL=1 sends
every patch to the latter).  Identical inverses make every sweep and every solve identical,
which is what is compared: one FP64 sweep per level on a seeded vector, and a whole solve.
"""
import os

import numpy as np
import pytest

import ib_workloads as W
from tests.gpu_helpers import host, torch_dev

pytestmark = pytest.mark.gpu


def _setup(api, rec, force_global, **kw):
    if force_global:
        os.environ["CAV_FACTOR_GLOBAL"] = "1"
    try:
        s = api.ib_setup(rec)
        h = api.cav_setup(s, **kw)
    finally:
        os.environ.pop("CAV_FACTOR_GLOBAL", None)
    return s, h


@pytest.mark.parametrize("name", ["membrane64", "membrane256", "beam128", "channel32"])
def test_pair_kernel_equals_global_kernel(name):
    from paper_2608_14310_b300 import api
    rec = {"membrane64": lambda: W.membrane_ellipse(64, 1e4),
           "membrane256": lambda: W.config2(256, 1e4),
           "beam128": lambda: W.beam_curve(128, 512, k_bend=1e3, k_stretch=1e5),
           "channel32": lambda: W.fiber_channel(32)}[name]()
    kw = dict(kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, alpha=0.85, precision="fp64")
    s1, h1 = _setup(api, rec, False, **kw)
    s2, h2 = _setup(api, rec, True, **kw)
    rng = np.random.default_rng(11)
    for l in range(api.cav_num_levels(h1) - 1):
        info = api.cav_get_level_info(h1, l)
        N = info["N"]
        b = rng.uniform(-1, 1, 3 * N * N)
        w0 = 1e-2 * rng.uniform(-1, 1, 3 * N * N)
        w1, w2 = torch_dev(w0), torch_dev(w0)
        api.cav_sweep(h1, l, torch_dev(b), w1)
        api.cav_sweep(h2, l, torch_dev(b), w2)
        assert np.array_equal(host(w1), host(w2)), (name, l, info["max_n"])
    b = rec.rhs()
    x1, x2 = torch_dev(np.zeros(b.size)), torch_dev(np.zeros(b.size))
    i1 = api.fgmres_solve(s1, h1, torch_dev(b), x1, rtol=1e-10, maxit=150, rel_to=1)
    i2 = api.fgmres_solve(s2, h2, torch_dev(b), x2, rtol=1e-10, maxit=150, rel_to=1)
    assert i1["iters"] == i2["iters"] and np.array_equal(host(x1), host(x2))
