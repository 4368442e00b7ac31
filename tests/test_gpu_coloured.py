"""GPU parity of the class-by-class multiplicative CAV sweep (Sec. 3.3) against the oracle,
through the C ABI, on the same seeded inputs:

  * colour classes: bit-exact with the oracle's first-fit colouring on every level;
  * one sweep per level: ||w_gpu - w_oracle|| / ||w_oracle|| <= the case's tolerance (1e-12
    for the plain FP64 target-point case; 1e-11 where the local matrices' condition number
    times eps separates the Gauss-Jordan and LU inverses, as for the additive sweep);
  * repeated sweeps give identical bits (no atomics, fixed reduction order);
  * one V-cycle within 10x the sweep tolerance; FGMRES iteration counts within one of the
    oracle's, both converged, solutions within 1e-8;
  * FP32 inverses: the FP64 FGMRES still reaches 1e-10 (true residual); BF16 inverses are
    refused at set-up (the undamped multiplicative sweep diverges with them, as the oracle
    shows).
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import colouring as ocol, fgmres as ofg, multigrid as omg
from tests.gpu_helpers import gpu_hierarchy, host, rel, torch_dev

pytestmark = pytest.mark.gpu

CASES = {
    "target32": (lambda: W.config1(), 2, 1e-12),
    "membrane32": (lambda: W.membrane_ellipse(32, 1e4), 1, 1e-11),
    "beam32": (lambda: W.beam_curve(32, 128, k_bend=1e-1, k_stretch=1e1), 1, 1e-11),
    "rows32": (lambda: W.paper_target_rows(32), 1, 1e-11),
    "nomarkers16": (lambda: W.System(name="empty", N=16, L=1.0, rho=1.0, mu=0.01, dt=0.01, law=0,
                                     closed=True, X=np.zeros((0, 2)), ds=0.1, omega=np.zeros(0)), 1, 1e-12),
}


class Pair:
    pass


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    mk, nu, tol = CASES[request.param]
    rec = mk()
    P = Pair()
    P.name, P.rec, P.nu, P.tol = request.param, rec, nu, tol
    P.levels = omg.build_hierarchy(rec, 8, "cav")
    P.sys, P.h = gpu_hierarchy(rec, kind="cav", coarsest_N=8, nu_pre=nu, nu_post=nu, precision="fp64",
                               smoother="coloured")
    return P


def test_colour_classes_bit_exact(pair):
    from paper_2608_14310_b300 import api
    for l, lev in enumerate(pair.levels[:-1]):
        want = omg.level_colours(lev)
        got = api.cav_colour_export(pair.h, l)
        assert np.array_equal(got, want), f"level {l}"
        assert api.cav_get_level_info(pair.h, l)["n_colours"] == int(want.max()) + 1


def test_one_coloured_sweep_per_level(pair):
    from paper_2608_14310_b300 import api
    rng = np.random.default_rng(23)
    worst = 0.0
    for l, lev in enumerate(pair.levels[:-1]):
        n = 3 * lev.N ** 2
        b = rng.uniform(-1, 1, n)
        b[2 * lev.N ** 2:] -= b[2 * lev.N ** 2:].mean()
        w0 = rng.uniform(-1, 1, n) * 1e-2
        w = torch_dev(w0)
        api.cav_sweep(pair.h, l, torch_dev(b), w)
        got = host(w)
        want = ocol.coloured_sweep(lev.KE, lev.solvers, omg.level_colours(lev), w0, b, lev.N)
        e = rel(got, want)
        worst = max(worst, e)
        assert e <= pair.tol, (l, e)
    print(f"{pair.name}: worst coloured sweep rel diff {worst:.3e}")


def test_coloured_sweep_is_deterministic(pair):
    from paper_2608_14310_b300 import api
    lev = pair.levels[0]
    b = W.rhs(lev.N, 5)
    outs = []
    for _ in range(3):
        w = torch_dev(np.full(b.size, 1e-3))
        api.cav_sweep(pair.h, 0, torch_dev(b), w)
        outs.append(host(w))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_coloured_vcycle(pair):
    from paper_2608_14310_b300 import api
    b = pair.rec.rhs()
    z = torch_dev(np.zeros(b.size))
    api.vcycle_apply(pair.h, torch_dev(b), z)
    want = omg.vcycle(pair.levels, b, pair.nu, pair.nu, "coloured")
    assert rel(host(z), want) <= 10 * pair.tol


def test_coloured_fgmres(pair):
    from paper_2608_14310_b300 import api
    b = pair.rec.rhs()
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(pair.sys, pair.h, torch_dev(b), x, rtol=1e-10, maxit=150)
    K = pair.levels[0].KE
    xo, io = ofg.fgmres(lambda v: K @ v, b,
                        lambda r: omg.vcycle(pair.levels, r, pair.nu, pair.nu, "coloured"),
                        rtol=1e-10, maxit=150)
    assert info["converged"] == 1 and io["converged"]
    assert abs(info["iters"] - io["iters"]) <= 1, (info["iters"], io["iters"])
    xg = host(x)
    assert np.linalg.norm(b - K @ xg) <= 2e-10 * np.linalg.norm(b)
    assert rel(xg, xo) <= 1e-8
    print(f"{pair.name}: coloured gpu its {info['iters']} oracle its {io['iters']} "
          f"relres {info['relres_true']:.2e}")


def test_coloured_rejects_bf16_inverses():
    from paper_2608_14310_b300 import api
    sys_ = api.ib_setup(W.membrane_ellipse(16, 1e4))
    with pytest.raises(api.IBError) as e:
        api.cav_setup(sys_, precision="bf16", smoother="coloured")
    assert e.value.status == api.IB_ERR_INVALID and "diverges" in str(e.value)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coloured_mixed_precision_reaches_tolerance(precision):
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(64, 1e4)
    sys_, h = gpu_hierarchy(rec, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, precision=precision,
                            smoother="coloured")
    b = rec.rhs()
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(sys_, h, torch_dev(b), x, rtol=1e-10, maxit=150)
    assert info["converged"] == 1 and info["relres_true"] <= 2e-10, info
    print(f"membrane64 coloured {precision}: {info['iters']} its, relres {info['relres_true']:.2e}")


def test_hybrid_vcycle_and_fgmres():
    # coloured (multiplicative) sweep on the finest level only, the weighted additive sweep
    # (two per side, alpha 0.85) on the coarser smoothing levels
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(32, 1e4)
    levels = omg.build_hierarchy(rec, 8, "cav")
    L = len(levels) - 1
    modes = ["coloured"] + ["additive"] * (L - 1)
    nus = [1] + [2] * (L - 1)
    sys_, h = gpu_hierarchy(rec, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, alpha=0.85, precision="fp64",
                            smoother="coloured", coloured_levels=1, nu_additive=2)
    infos = [api.cav_get_level_info(h, l) for l in range(L)]
    assert infos[0]["n_colours"] > 0 and all(i["n_colours"] == 0 for i in infos[1:])
    b = rec.rhs()
    z = torch_dev(np.zeros(b.size))
    api.vcycle_apply(h, torch_dev(b), z)
    want = omg.vcycle(levels, b, nus, nus, modes, 0.85)
    assert rel(host(z), want) <= 1e-10
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(sys_, h, torch_dev(b), x, rtol=1e-10, maxit=150)
    K = levels[0].KE
    _, io = ofg.fgmres(lambda v: K @ v, b, lambda r: omg.vcycle(levels, r, nus, nus, modes, 0.85),
                       rtol=1e-10, maxit=150)
    assert info["converged"] == 1 and io["converged"]
    assert abs(info["iters"] - io["iters"]) <= 1, (info["iters"], io["iters"])
    print(f"membrane32 hybrid: gpu its {info['iters']} oracle its {io['iters']}")


def test_diverging_fp32_multiplicative_sweep_stops_cleanly():
    # the stiff N = 512 beam (bending 1e3, stretching 1e5): its enlarged patches' condition
    # numbers reach about 1e10, so FP32-rounded inverses make the undamped coloured sweep
    # diverge; FGMRES stops at the first non-finite residual estimate, says why, and returns
    # the last finite iterate instead of NaN
    from paper_2608_14310_b300 import api
    rec = W.config3()
    sys_, h = gpu_hierarchy(rec, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, precision="fp32",
                            smoother="coloured")
    b = rec.rhs()
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(sys_, h, torch_dev(b), x, rtol=1e-10, maxit=20)
    assert info["converged"] == 0 and info["iters"] < 20, info
    assert "not finite" in api._lib.ib_last_error().decode()
    assert np.isfinite(host(x)).all()


@pytest.mark.parametrize("nu_pre,nu_post", [(1, 0), (0, 1)])
def test_hybrid_vcycle_with_one_sided_finest_smoothing(nu_pre, nu_post):
    # the same hybrid V-cycle with sweeps on one side of the finest level only: with no
    # post-sweep the cycle's output is the pre-smoothed iterate plus the prolonged correction,
    # whose pressure mean the oracle's coarse levels removed after each of their sweeps
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(32, 1e4)
    levels = omg.build_hierarchy(rec, 8, "cav")
    L = len(levels) - 1
    modes = ["coloured"] + ["additive"] * (L - 1)
    pre = [nu_pre] + [2] * (L - 1)
    post = [nu_post] + [2] * (L - 1)
    sys_, h = gpu_hierarchy(rec, kind="cav", coarsest_N=8, nu_pre=nu_pre, nu_post=nu_post, alpha=0.85,
                            precision="fp64", smoother="coloured", coloured_levels=1, nu_additive=2)
    b = rec.rhs()
    z = torch_dev(np.zeros(b.size))
    api.vcycle_apply(h, torch_dev(b), z)
    want = omg.vcycle(levels, b, pre, post, modes, 0.85)
    assert rel(host(z), want) <= 1e-10
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(sys_, h, torch_dev(b), x, rtol=1e-10, maxit=150)
    K = levels[0].KE
    _, io = ofg.fgmres(lambda v: K @ v, b, lambda r: omg.vcycle(levels, r, pre, post, modes, 0.85),
                       rtol=1e-10, maxit=150)
    assert info["converged"] == 1 and io["converged"]
    assert abs(info["iters"] - io["iters"]) <= 1, (info["iters"], io["iters"])
    print(f"membrane32 hybrid {nu_pre}+{nu_post}: gpu its {info['iters']} oracle its {io['iters']}")
