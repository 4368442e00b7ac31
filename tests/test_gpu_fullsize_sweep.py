"""Whole-vector sweep parity at the bench's size: the elliptic membrane at N = 256 (1024
markers, kappa_s = 1e4, config 2), in the launch configuration the bench uses (weighted
additive CAV, alpha 0.85, autotuned patch-apply variants), against the oracle's
additive_sweep on every smoothing level (256, 128, 64, 32, 16), element by element.

  * FP64 inverses: ||w_gpu - w_oracle|| / ||w_oracle|| <= 1e-12 per sweep, the plain path's
    bound;
  * FP32 inverses (the bench's headline precision): the correction w - w0 within 1e-5
    relative of the oracle's FP64 correction -- the storage rounding of the equilibrated
    inverses (unit roundoff 2^-24) amplified by the patch solve, as in the small-size
    mixed-precision tests.

The oracle hierarchy with its 65,536 factorised patches per finest level takes about a
minute to build on one core.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import multigrid as omg, smoother as osm
from tests.gpu_helpers import host, rel, torch_dev

pytestmark = pytest.mark.gpu

ALPHA = 0.85
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def membrane256():
    from paper_2608_14310_b300 import api
    rec = W.config2(256, 1e4)
    levels = omg.build_hierarchy(rec, 8, "cav")
    sysm = api.ib_setup(rec)
    hs = {p: api.cav_setup(sysm, nu_pre=2, nu_post=2, alpha=ALPHA, precision=p, autotune=True)
          for p in ("fp64", "fp32")}
    return rec, levels, sysm, hs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_whole_sweep_every_level(membrane256, precision):
    from paper_2608_14310_b300 import api
    rec, levels, sysm, hs = membrane256
    h = hs[precision]
    assert api.cav_num_levels(h) == len(levels)
    rng = np.random.default_rng(41)
    worst = []
    for l, lev in enumerate(levels[:-1]):
        N = lev.N
        n = 3 * N * N
        b = rng.uniform(-1, 1, n)
        b[2 * N * N:] -= b[2 * N * N:].mean()
        w0 = rng.uniform(-1, 1, n) * 1e-2
        w = torch_dev(w0)
        api.cav_sweep(h, l, torch_dev(b), w)
        got = host(w)
        want = osm.additive_sweep(lev.KE, lev.solvers, lev.theta, w0, b, N, ALPHA)
        e = rel(got, want) if precision == "fp64" else rel(got - w0, want - w0)
        worst.append(e)
        assert e <= TOL[precision], (l, N, e)
    print(f"membrane256 {precision}: per-level sweep rel diff " + ", ".join(f"{e:.2e}" for e in worst))
