"""Mixed precision (enlarged-patch inverses stored in FP32 or BF16, FP32 accumulation;
everything else FP64) against the FP64 oracle.

Tolerances from the arithmetic: one sweep's correction differs from the FP64 one by the
storage rounding of the equilibrated inverse (unit roundoff 2^-24 for FP32, 2^-8 for BF16)
amplified by the patch solve, so the sweep is compared at 1e-5 (FP32) and 5e-2 (BF16)
relative; the preconditioner only has to be a preconditioner, so FGMRES must still reach
the 1e-10 relative residual in FP64 and agree with the oracle's FP64 solution to 1e-7.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import fgmres as ofg, multigrid as omg, smoother as osm
from tests.gpu_helpers import gpu_hierarchy, host, rel, torch_dev

pytestmark = pytest.mark.gpu

ALPHA = 0.85
SWEEP_TOL = {"fp32": 1e-5, "bf16": 5e-2}
CASES = {
    "membrane32": lambda: W.membrane_ellipse(32, 1e4),
    "beam32": lambda: W.beam_curve(32, 128, k_bend=1e-1, k_stretch=1e1),
    "target32": lambda: W.config1(),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def oracle_case(request):
    rec = CASES[request.param]()
    return request.param, rec, omg.build_hierarchy(rec, 8, "cav")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mixed_sweep_and_solve(oracle_case, precision):
    from paper_2608_14310_b300 import api
    name, rec, levels = oracle_case
    sysm, h = gpu_hierarchy(rec, nu_pre=2, nu_post=2, alpha=ALPHA, precision=precision)
    info0 = api.cav_get_level_info(h, 0)
    s = {"fp32": 4, "bf16": 2}[precision]
    assert info0["inverse_bytes"] == s * sum(((n + 7) // 8 * 8) * n for n in
                                             [len(p) for p in levels[0].patches if len(p) > 5])
    rng = np.random.default_rng(21)
    lev = levels[0]
    n = 3 * lev.N ** 2
    b = rng.uniform(-1, 1, n)
    w0 = rng.uniform(-1, 1, n) * 1e-2
    w = torch_dev(w0)
    api.cav_sweep(h, 0, torch_dev(b), w)
    want = osm.additive_sweep(lev.KE, lev.solvers, lev.theta, w0, b, lev.N, ALPHA)
    e_sweep = rel(host(w) - w0, want - w0)
    assert e_sweep <= SWEEP_TOL[precision], e_sweep
    b = rec.rhs()
    x = torch_dev(np.zeros(n))
    info = api.fgmres_solve(sysm, h, torch_dev(b), x, rtol=1e-10, maxit=150)
    assert info["converged"] == 1, info
    K = lev.KE
    xg = host(x)
    assert np.linalg.norm(b - K @ xg) <= 2e-10 * np.linalg.norm(b)
    xo, io = ofg.fgmres(lambda v: K @ v, b, lambda r: omg.vcycle(levels, r, 2, 2, "additive", ALPHA),
                        rtol=1e-10, maxit=150)
    e_sol = rel(xg, xo)
    assert e_sol <= 1e-7, e_sol
    print(f"{name} {precision}: sweep corr rel diff {e_sweep:.2e}, its {info['iters']} (oracle fp64 "
          f"{io['iters']}), relres {info['relres_true']:.2e}, |x-x_oracle|/|x| {e_sol:.2e}")
