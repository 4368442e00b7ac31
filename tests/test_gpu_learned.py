"""Time stepping and the learned initial guess.

* the step's pieces (E X + k_t X_target, S F, J u, the right-hand side of Eq. Eul_schur, the
  marker update of Eq. im_disc_advec) against the oracle, to 1e-13 relative;
* the network's forward pass, loss and every parameter gradient against the FP64 oracle
  (oracle/cnn.py, itself pinned by finite differences): FP32 kernels, so outputs and loss to
  1e-5 relative, gradients to 2e-4 of each layer's largest gradient;
* the pack / apply kernels against their definitions;
* training on the GPU lowers the loss, and the trained network's guesses need fewer FGMRES
  iterations than the previous-step guess on held-out steps, every solve still reaching 1e-10.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import cnn, ib as oib
from tests.gpu_helpers import host, torch_dev

pytestmark = pytest.mark.gpu


def _perturbed_ring(N=32):
    rec = W.tethered_ring(N)
    rng = np.random.default_rng(4)
    rec.X = rec.X + rng.uniform(-0.3, 0.3, rec.X.shape) / N
    return rec


def test_step_pieces_match_oracle():
    import torch
    from paper_2608_14310_b300 import api
    rec = _perturbed_ring()
    N, M = rec.N, rec.M
    s = api.ib_setup(rec)
    F = torch.empty(2 * M, dtype=torch.float64, device="cuda")
    api.ib_force(s, F)
    Fo = oib.force_vector(rec)
    assert np.abs(host(F) - Fo).max() <= 1e-13 * np.abs(Fo).max()
    f = torch.empty(2 * N * N, dtype=torch.float64, device="cuda")
    api.ib_spread(s, F, f)
    S = oib.spreading_matrix(N, rec.h, rec.X, rec.omega)
    fo = S @ Fo
    assert np.abs(host(f) - fo).max() <= 1e-13 * np.abs(fo).max()
    rng = np.random.default_rng(5)
    u = rng.standard_normal(3 * N * N)
    U = torch.empty(2 * M, dtype=torch.float64, device="cuda")
    api.ib_interp(s, torch_dev(u), U)
    Uo = oib.interpolation_matrix(N, rec.h, rec.X) @ u[:2 * N * N]
    assert np.abs(host(U) - Uo).max() <= 1e-13 * np.abs(Uo).max()
    fb = W.shear_forcing(N, 0.1)
    b = torch.empty(3 * N * N, dtype=torch.float64, device="cuda")
    api.ib_step_rhs(s, torch_dev(u), torch_dev(fb), b)
    bo = oib.step_rhs(rec, u, fb)
    assert np.abs(host(b) - bo).max() <= 1e-13 * np.abs(bo).max()
    Xn = api.ib_advect(s, torch_dev(u))
    assert np.abs(Xn - oib.advect(rec, u)).max() <= 1e-15


def test_network_forward_and_gradients_match_oracle():
    import torch
    from paper_2608_14310_b300 import api
    dims = dict(in_ch=15, hidden=8, n_hidden=2, out_ch=3)
    net = api.IBNet(15, 8, 2, 3, seed=3)
    B, N = 2, 16
    rng = np.random.default_rng(6)
    x = rng.standard_normal((B, 15, N, N)).astype(np.float32)
    t = rng.standard_normal((B, 3, N, N)).astype(np.float32)
    xd = torch.from_numpy(x.ravel().copy()).cuda()
    td = torch.from_numpy(t.ravel().copy()).cuda()
    out = torch.empty(B * 3 * N * N, dtype=torch.float32, device="cuda")
    net.forward(xd, out, B, N)
    p = net.get_params().astype(np.float64)
    lo, go, oo = cnn.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64), **dims)
    og = host(out).reshape(B, 3, N, N)
    assert np.abs(og - oo).max() <= 1e-5 * np.abs(oo).max()
    loss, g = net.gradients(xd, td, B, N)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    cin, cout = cnn.layer_shapes(**dims)
    off = 0
    for ci, co in zip(cin, cout):
        for n in (co * ci * 9, co):
            gs, os_ = g[off:off + n], go[off:off + n]
            assert np.abs(gs - os_).max() <= 2e-4 * np.abs(os_).max() + 1e-12, (off, n)
            off += n


def test_pack_and_apply_kernels():
    import torch
    from paper_2608_14310_b300 import api
    N = 12
    NN = N * N
    rng = np.random.default_rng(8)
    xs = [rng.standard_normal(3 * NN) for _ in range(3)]
    fs = [rng.standard_normal(2 * NN) for _ in range(3)]
    sc = list(rng.uniform(0.5, 2.0, 15))
    out = torch.empty(15 * NN, dtype=torch.float32, device="cuda")
    api.ibnet_pack_input(N, [torch_dev(a) for a in xs], [torch_dev(a) for a in fs], sc, out)
    def field(t, k):
        return xs[t][k * NN:(k + 1) * NN] if k < 3 else fs[t][(k - 3) * NN:(k - 2) * NN]
    want = np.concatenate([np.concatenate([field(t + 1, k) - field(t, k) if t < 2 else field(2, k)
                                           for k in range(5)]) for t in range(3)])
    want = want / np.repeat(np.array(sc), NN)
    assert np.allclose(host(out), (want / 1.0).astype(np.float32), rtol=1e-6, atol=1e-7)
    osc = [2.0, 0.5, 3.0]
    tg = torch.empty(3 * NN, dtype=torch.float32, device="cuda")
    api.ibnet_pack_target(N, torch_dev(xs[1]), torch_dev(xs[0]), osc, tg)
    assert np.allclose(host(tg), ((xs[1] - xs[0]) / np.repeat(osc, NN)).astype(np.float32), rtol=1e-6)
    api.ibnet_pack_target(N, torch_dev(xs[2]), torch_dev(xs[1]), osc, tg, x_prev2=torch_dev(xs[0]))
    want = (xs[2] - 2 * xs[1] + xs[0]) / np.repeat(osc, NN)
    assert np.allclose(host(tg), want.astype(np.float32), rtol=1e-6, atol=1e-7)
    d = torch.from_numpy(rng.standard_normal(3 * NN).astype(np.float32)).cuda()
    g = torch.empty(3 * NN, dtype=torch.float64, device="cuda")
    api.ibnet_apply_delta(N, torch_dev(xs[2]), d, osc, g)
    assert np.allclose(host(g), xs[2] + np.repeat(osc, NN) * host(d).astype(np.float64), rtol=1e-12)
    api.ibnet_apply_delta(N, torch_dev(xs[2]), d, osc, g, x_prev2=torch_dev(xs[1]))
    want = 2 * xs[2] - xs[1] + np.repeat(osc, NN) * host(d).astype(np.float64)
    assert np.allclose(host(g), want, rtol=1e-12, atol=1e-14)
    # quadratic extrapolation base 3 x2 - 3 x1 + x0 (a fourth step as the new value)
    x3 = rng.standard_normal(3 * NN)
    api.ibnet_pack_target(N, torch_dev(x3), torch_dev(xs[2]), osc, tg, x_prev2=torch_dev(xs[1]),
                          x_prev3=torch_dev(xs[0]))
    want = (x3 - (3 * xs[2] - 3 * xs[1] + xs[0])) / np.repeat(osc, NN)
    assert np.allclose(host(tg), want.astype(np.float32), rtol=1e-6, atol=1e-6)
    api.ibnet_apply_delta(N, torch_dev(xs[2]), d, osc, g, x_prev2=torch_dev(xs[1]), x_prev3=torch_dev(xs[0]))
    want = 3 * xs[2] - 3 * xs[1] + xs[0] + np.repeat(osc, NN) * host(d).astype(np.float64)
    assert np.allclose(host(g), want, rtol=1e-12, atol=1e-13)


def test_training_lowers_loss():
    import torch
    from paper_2608_14310_b300 import api
    net = api.IBNet(15, 16, 2, 3, seed=5)
    B, N = 4, 16
    rng = np.random.default_rng(9)
    x = torch.from_numpy(rng.standard_normal(B * 15 * N * N).astype(np.float32)).cuda()
    # a learnable target: a fixed linear map of the input channels
    xa = host(x).reshape(B, 15, N, N)
    t = (0.5 * xa[:, 10:13] - 0.25 * xa[:, 5:8]).astype(np.float32)
    td = torch.from_numpy(t.ravel().copy()).cuda()
    first = net.train_step(x, td, B, N, 3e-3, want_loss=True)
    for _ in range(150):
        last = net.train_step(x, td, B, N, 3e-3, want_loss=True)
    assert last < 0.3 * first, (first, last)


def test_learned_guess_saves_iterations():
    from paper_2608_14310_b300.learned_guess import LearnedGuess, TimeSeries
    rec = W.tethered_ring(32, dt_factor=0.25)
    ts = TimeSeries(rec, W.shear_forcing, nu=2, alpha=0.85, precision="fp32")
    n_train, n_fit, n_test = 180, 160, 60
    for _ in range(n_train):
        ts.step()
    lg = LearnedGuess(rec.N, hidden=32, n_hidden=3)
    lg.fit_scales(ts, n_fit)
    info = lg.train(ts, n_fit, iters=800, batch=16, lr=1e-3)
    assert info["losses"][-1][1] < info["losses"][0][1]
    cal = lg.calibrate(ts, n_fit, n_train)
    assert all(0.0 <= g <= 1.0 for g in cal["gamma"])
    # on the held-out steps the calibrated correction is never worse than none (gamma = 0)
    assert all(c <= 1.0 + 1e-9 for c in cal["heldout_rel_sq_error_calibrated"]), cal
    res = {"learned": [], "extrapolated": [], "previous": []}
    for _ in range(n_test):
        out = ts.step(guesses=(("learned", lambda s: lg.predict(s)), ("extrapolated", lambda s: lg.extrapolate(s)),
                               ("previous", None)))
        for lab, inf, _ in out:
            assert inf["converged"] == 1
            res[lab].append((inf["iters"], inf["r0"]))
    m = {k: (np.mean([a for a, _ in v]), np.exp(np.mean(np.log([b for _, b in v])))) for k, v in res.items()}
    print("learned guess: " + ", ".join(f"{k}: mean iters {a:.2f}, geo-mean r0 {b:.2e}" for k, (a, b) in m.items())
          + f"; loss {info['losses'][0][1]:.3e} -> {info['losses'][-1][1]:.3e}; calibration {cal}")
    # the network's guess starts closer than the previous-step guess and needs fewer iterations
    assert m["learned"][1] < m["previous"][1]
    assert m["learned"][0] < m["previous"][0]
    # and, calibrated on held-out steps, it does not start farther than the extrapolation it corrects
    assert m["learned"][1] <= 1.05 * m["extrapolated"][1], m
    assert m["learned"][0] <= m["extrapolated"][0] + 0.5, m


def test_learned_guess_on_the_fiber_channel():
    """The fiber benchmark's time loop (Sec. 5.3, a short run at N = 16): the CNN corrects the
    quadratic extrapolation from the last four steps; calibrated on held-out steps it starts
    each step's Newton solve no farther than that extrapolation and much closer than the
    previous step's solution, and saves FGMRES iterations over the latter."""
    from paper_2608_14310_b300.learned_guess import ChannelSeries, LearnedGuess
    rec = W.fiber_channel(16)
    cs = ChannelSeries(rec, cav=dict(kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, smoother="coloured",
                                     precision="fp64"))
    n_train, n_fit, n_test = 300, 270, 40
    for _ in range(n_train):
        cs.step()
    lg = LearnedGuess(rec.N, hidden=16, n_hidden=2, base="quadratic", history=4)
    lg.fit_scales(cs, n_fit, start=120)
    lg.train(cs, n_fit, iters=600, batch=16, lr=1e-3, start=120)
    cal = lg.calibrate(cs, n_fit, n_train)
    assert all(c <= 1.0 + 1e-9 for c in cal["heldout_rel_sq_error_calibrated"]), cal
    cal.update(lg.calibrate_residual(cs, n_fit, n_train, stride=3))
    # the search keeps the best scale it tried: never worse than the base on the held-out steps
    assert cal["heldout_first_residual_geomean"] <= cal["heldout_first_residual_geomean_base"] * (1 + 1e-12), cal
    variants = (("learned", lambda s: lg.predict(s), "fp64"), ("quadratic", lambda s: lg.extrapolate(s, 2), "fp64"),
                ("previous", None, "fp64"))
    res = {v[0]: [] for v in variants}
    for _ in range(n_test):
        for lab, inf in cs.step(variants):
            assert inf["converged"]
            res[lab].append(inf)
    r0 = {k: float(np.exp(np.mean(np.log([max(r["r0"], 1e-300) for r in v])))) for k, v in res.items()}
    it = {k: float(np.mean([r["fgmres_total"] for r in v])) for k, v in res.items()}
    print(f"fiber channel N=16: first residual {r0}, FGMRES per step {it}, calibration {cal}")
    assert r0["learned"] < 0.1 * r0["previous"] and it["learned"] < it["previous"]
    assert r0["learned"] <= 1.05 * r0["quadratic"], (r0, cal)
