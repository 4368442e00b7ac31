"""Time-stepped solves of the reduced IB system with a learned initial guess.

Each step n builds S^n, J^n and E_E at the markers' configuration X^n, rebuilds the CAV
hierarchy, forms the right-hand side of Eq. (Eul_schur) for the semi-implicit step
(Eq. im_disc_mom without convection), solves with CAV-preconditioned FGMRES to a relative
residual of rtol (relative to ||b||), and advances the markers by Eq. (im_disc_advec).
The initial guess is either the previous step's solution or the prediction of a small CNN
(library's ibnet) from the previous three steps' solutions and spread Lagrangian forces.
Every numerical step runs in the CUDA library; this module only sequences calls and moves
buffers.
"""
from __future__ import annotations

import math
import time
from dataclasses import replace

import numpy as np

from . import api


class TimeSeries:
    """Run the time stepping, keeping every step's solution and spread force on the device."""

    def __init__(self, rec, forcing, nu=2, alpha=0.85, precision="fp32", rtol=1e-10, maxit=150,
                 autotune=False):
        import torch
        self.torch = torch
        self.rec0 = rec
        self.forcing = forcing
        self.kw = dict(nu_pre=nu, nu_post=nu, alpha=alpha, precision=precision, autotune=autotune,
                       krylov_capacity=maxit)
        self.rtol, self.maxit = rtol, maxit
        self.N = rec.N
        self.n = 3 * rec.N * rec.N
        self.X = np.array(rec.X, dtype=np.float64)
        self.x_hist = []   # solutions x^1, x^2, ... (device, float64, 3N^2)
        self.f_hist = []   # spread forces f^0, f^1, ... (device, float64, 2N^2)
        self.records = []  # per step: iterations, solve ms, converged, which guess
        x0 = torch.zeros(self.n, dtype=torch.float64, device="cuda")
        self.x_hist.append(x0)          # x^0 = 0 (fluid at rest)

    def _system(self):
        rec = replace(self.rec0, X=self.X.copy())
        return api.ib_setup(rec)

    def step(self, guesses=(("previous", None),)):
        """One time step.  guesses: (label, fn[, precision]) entries; fn(self) returns an initial
        guess (device vector) once this step's force is stored, or fn is None for the previous
        solution x^n; precision (default: the series') selects the stored-inverse precision of
        the hierarchy used for that solve.  The same system is solved from every entry; the
        first one's solution advances the series, the others are for comparison.  Returns the
        list of (label, info, ms); ms covers the solve only (hierarchies are rebuilt per step)."""
        torch = self.torch
        n_step = len(self.x_hist) - 1
        sysm = self._system()
        hier = {}
        N = self.N
        F = torch.empty(2 * self.rec0.M, dtype=torch.float64, device="cuda")
        api.ib_force(sysm, F)
        f = torch.empty(2 * N * N, dtype=torch.float64, device="cuda")
        api.ib_spread(sysm, F, f)
        self.f_hist.append(f)
        fb = torch.from_numpy(self.forcing(N, n_step * self.rec0.dt)).cuda()
        b = torch.empty(self.n, dtype=torch.float64, device="cuda")
        api.ib_step_rhs(sysm, self.x_hist[-1], fb, b)
        out = []
        x_main = None
        for entry in guesses:
            label, fn = entry[0], entry[1]
            prec = entry[2] if len(entry) > 2 else self.kw["precision"]
            if prec not in hier:
                hier[prec] = api.cav_setup(sysm, **dict(self.kw, precision=prec))
            h = hier[prec]
            x = (self.x_hist[-1] if fn is None else fn(self)).clone()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            info = api.fgmres_solve(sysm, h, b, x, rtol=self.rtol, maxit=self.maxit, history=True)
            info["r0"] = float(info["history"][0])  # ||b - K x_guess|| / ||b||
            ev1.record()
            torch.cuda.synchronize()
            out.append((label, info, ev0.elapsed_time(ev1)))
            if x_main is None:
                x_main = x
        self.x_hist.append(x_main)
        self.X = api.ib_advect(sysm, x_main)
        self.records.append(out)
        for h in hier.values():
            h.close()
        sysm.close()
        return out


class LearnedGuess:
    """The CNN and its normalisation, trained on a TimeSeries' stored steps."""

    def __init__(self, N, hidden=32, n_hidden=3, seed=7, base: str = "linear", history: int = 3):
        """base: the extrapolation the network corrects, "linear" (2 x^n - x^{n-1}) or
        "quadratic" (3 x^n - 3 x^{n-1} + x^{n-2}).  history: 3, the last three steps as two
        increments and the newest fields (15 channels); or 4, the last four steps as their
        backward differences in time of order 3, 2, 1, 0 at the newest step (20 channels)."""
        import torch
        assert base in ("linear", "quadratic") and history in (3, 4)
        self.torch = torch
        self.N = N
        self.base = base
        self.history = history
        self.in_ch = 5 * history
        self.net = api.IBNet(self.in_ch, hidden, n_hidden, 3, seed)
        self.in_scale = None
        self.out_scale = None
        self.gamma = [1.0, 1.0, 1.0]   # per-field scale of the correction (calibrate)

    def _hist(self, ts, i):
        # x_prev2 and x_prev3 of the base extrapolation from step i
        if self.base == "quadratic":
            return dict(x_prev2=ts.x_hist[i - 1], x_prev3=ts.x_hist[i - 2])
        return dict(x_prev2=ts.x_hist[i - 1])

    def fit_scales(self, ts: TimeSeries, upto: int, start: int = 0):
        """Per-channel RMS of the training range [start, upto) (host statistics of a few
        sampled steps; upto = number of completed steps, so x^{i+1} and f^i exist for i < upto)."""
        N = self.N
        NN = N * N
        first = max(start, self.history - 1, 2)
        idx = np.linspace(first, upto - 1, num=min(16, max(1, upto - first)), dtype=int)
        xs = np.stack([ts.x_hist[i].cpu().numpy() for i in idx])
        fs = np.stack([ts.f_hist[i].cpu().numpy() for i in idx])
        dx = np.stack([(ts.x_hist[i + 1] - ts.x_hist[i]).cpu().numpy() for i in idx])
        if self.base == "quadratic":
            d2x = np.stack([(ts.x_hist[i + 1] - 3 * ts.x_hist[i] + 3 * ts.x_hist[i - 1] - ts.x_hist[i - 2]).cpu().numpy()
                            for i in idx])
        else:
            d2x = np.stack([(ts.x_hist[i + 1] - 2 * ts.x_hist[i] + ts.x_hist[i - 1]).cpu().numpy() for i in idx])
        rms = lambda a: float(np.sqrt(np.mean(a * a))) or 1.0  # noqa: E731
        dfs = np.stack([(ts.f_hist[i] - ts.f_hist[i - 1]).cpu().numpy() for i in idx])
        fields_x = [rms(xs[:, k * NN:(k + 1) * NN]) for k in range(3)]
        fields_f = [rms(fs[:, k * NN:(k + 1) * NN]) for k in range(2)]
        incr_x = [rms(dx[:, k * NN:(k + 1) * NN]) for k in range(3)]
        incr_f = [rms(dfs[:, k * NN:(k + 1) * NN]) for k in range(2)]
        if self.history == 3:
            # channel groups: increments (two steps), then the current state
            self.in_scale = (incr_x + incr_f) * 2 + fields_x + fields_f
        else:
            # differences of order 3, 2, 1 in time at step i, then the current state
            def diff(h, i, d):
                c, v = 1.0, 0
                for m in range(d + 1):
                    v = v + c * h[i - m]
                    c = -c * (d - m) / (m + 1)
                return v.cpu().numpy()
            sc = []
            for d in (3, 2):
                dxd = np.stack([diff(ts.x_hist, i, d) for i in idx if i >= 3])
                dfd = np.stack([diff(ts.f_hist, i, d) for i in idx if i >= 3])
                sc += [rms(dxd[:, k * NN:(k + 1) * NN]) for k in range(3)]
                sc += [rms(dfd[:, k * NN:(k + 1) * NN]) for k in range(2)]
            self.in_scale = sc + incr_x + incr_f + fields_x + fields_f
        # the network predicts the correction to the base extrapolation
        self.out_scale = [rms(d2x[:, k * NN:(k + 1) * NN]) for k in range(3)]

    def _pack(self, ts, i, out):
        # inputs from the last `history` steps up to i (solutions and spread forces)
        if self.history == 3:
            api.ibnet_pack_input(self.N, [ts.x_hist[i - 2], ts.x_hist[i - 1], ts.x_hist[i]],
                                 [ts.f_hist[i - 2], ts.f_hist[i - 1], ts.f_hist[i]], self.in_scale, out)
        else:
            api.ibnet_pack_history(self.N, [ts.x_hist[i - q] for q in (3, 2, 1, 0)],
                                   [ts.f_hist[i - q] for q in (3, 2, 1, 0)], self.in_scale, out)

    def train(self, ts: TimeSeries, upto: int, iters=1500, batch=16, lr=1e-3, seed=11, start: int = 0):
        torch = self.torch
        N = self.N
        NN = N * N
        samples = np.arange(max(start, self.history - 1), upto)   # x^{i+1} must exist: i + 1 <= upto
        C = self.in_ch
        xin = torch.empty(batch * C * NN, dtype=torch.float32, device="cuda")
        tgt = torch.empty(batch * 3 * NN, dtype=torch.float32, device="cuda")
        rng = np.random.default_rng(seed)
        losses = []
        t0 = time.perf_counter()
        for it in range(iters):
            pick = rng.choice(samples, batch, replace=len(samples) < batch)
            for s, i in enumerate(pick):
                self._pack(ts, int(i), xin[s * C * NN:(s + 1) * C * NN])
                api.ibnet_pack_target(N, ts.x_hist[int(i) + 1], ts.x_hist[int(i)], self.out_scale,
                                      tgt[s * 3 * NN:(s + 1) * 3 * NN], **self._hist(ts, int(i)))
            step_lr = lr * (0.5 * (1 + math.cos(math.pi * it / iters)) * 0.9 + 0.1)
            want = (it % 50 == 0) or it == iters - 1
            loss = self.net.train_step(xin, tgt, batch, N, step_lr, want_loss=want)
            if want:
                losses.append((it, loss))
        torch.cuda.synchronize()
        return {"losses": losses, "train_s": time.perf_counter() - t0}

    def calibrate(self, ts: TimeSeries, lo: int, hi: int):
        """Per field (u, v, p), the least-squares scale gamma of the network's correction on the
        held-out steps [lo, hi) (not used in training): gamma_f = <d_f, t_f> / <d_f, d_f> with d
        the network's output and t the true correction (both in the scaled units of training),
        clamped to [0, 1].  A correction that does not generalise is damped towards the
        extrapolation it corrects instead of adding its error to it."""
        torch = self.torch
        N = self.N
        NN = N * N
        xin = torch.empty(self.in_ch * NN, dtype=torch.float32, device="cuda")
        d = torch.empty(3 * NN, dtype=torch.float32, device="cuda")
        t = torch.empty(3 * NN, dtype=torch.float32, device="cuda")
        dt_, dd_, tt_ = np.zeros(3), np.zeros(3), np.zeros(3)
        for i in range(max(lo, self.history - 1), hi):
            self._pack(ts, i, xin)
            self.net.forward(xin, d, 1, N)
            api.ibnet_pack_target(N, ts.x_hist[i + 1], ts.x_hist[i], self.out_scale, t, **self._hist(ts, i))
            for f in range(3):
                df, tf = d[f * NN:(f + 1) * NN], t[f * NN:(f + 1) * NN]
                dt_[f] += self.net.inner(df, tf)
                dd_[f] += self.net.inner(df, df)
                tt_[f] += self.net.inner(tf, tf)
        self.gamma = [float(min(1.0, max(0.0, dt_[f] / dd_[f]))) if dd_[f] > 0 else 0.0 for f in range(3)]
        # relative error of the correction on the held-out steps: raw network and calibrated
        raw = [float((dd_[f] - 2 * dt_[f] + tt_[f]) / tt_[f]) if tt_[f] > 0 else 0.0 for f in range(3)]
        g = self.gamma
        cal = [float((g[f] ** 2 * dd_[f] - 2 * g[f] * dt_[f] + tt_[f]) / tt_[f]) if tt_[f] > 0 else 0.0
               for f in range(3)]
        return {"gamma": self.gamma, "heldout_rel_sq_error_raw": raw, "heldout_rel_sq_error_calibrated": cal,
                "heldout_steps": [lo, hi]}

    def start_online(self, ts, lo: int, hi: int, forget: float = 0.9):
        """Start the online scale: per field, exponentially weighted sums of <d, t> and <d, d> over
        the solved steps (weight `forget` per step), seeded with the steps [lo, hi); observe()
        adds each newly solved step, and predict(..., online=True) uses the current ratio."""
        self.forget = forget
        self.sdt, self.sdd = np.zeros(3), np.zeros(3)
        for i in range(max(lo, self.history - 1), hi):
            self._accumulate(ts, i)

    def _accumulate(self, ts, i: int):
        torch = self.torch
        N = self.N
        NN = N * N
        xin = torch.empty(self.in_ch * NN, dtype=torch.float32, device="cuda")
        d = torch.empty(3 * NN, dtype=torch.float32, device="cuda")
        t = torch.empty(3 * NN, dtype=torch.float32, device="cuda")
        self._pack(ts, i, xin)
        self.net.forward(xin, d, 1, N)
        api.ibnet_pack_target(N, ts.x_hist[i + 1], ts.x_hist[i], self.out_scale, t, **self._hist(ts, i))
        for f in range(3):
            df, tf = d[f * NN:(f + 1) * NN], t[f * NN:(f + 1) * NN]
            self.sdt[f] = self.forget * self.sdt[f] + self.net.inner(df, tf)
            self.sdd[f] = self.forget * self.sdd[f] + self.net.inner(df, df)

    def observe(self, ts):
        """After a step is solved: add it (the step from x^{n-1} to x^n, the newest stored)."""
        self._accumulate(ts, len(ts.x_hist) - 2)

    def online_gamma(self):
        return [float(min(1.0, max(0.0, self.sdt[f] / self.sdd[f]))) if self.sdd[f] > 0 else 0.0 for f in range(3)]

    def calibrate_residual(self, cs, lo: int, hi: int, stride: int = 5, grid=(0.0, 0.25, 0.5, 0.75, 1.0),
                           sweeps: int = 2):
        """For a ChannelSeries: per field, the scale gamma of the correction that minimises the
        geometric mean of the first Newton residual over the held-out steps lo, lo + stride, ...
        < hi (each re-evaluated from its stored state, `ChannelSeries.first_residual`), by
        coordinate search over `grid`, starting from the better of the least-squares fit
        (calibrate) and no correction, so the result is never worse than the base there.  The first
        residual weighs a velocity error's divergence, which the least-squares fit does not see."""
        steps = [i for i in range(max(lo, self.history - 1), hi, stride)]

        def score(gm):
            return float(np.mean([np.log(max(cs.first_residual(i, self.predict(cs, i=i, gamma=gm)), 1e-300))
                                  for i in steps]))

        base_s = score([0.0, 0.0, 0.0])
        start_s = score(list(self.gamma))
        best, best_s = (list(self.gamma), start_s) if start_s <= base_s else ([0.0, 0.0, 0.0], base_s)
        for _ in range(sweeps):
            for f in range(3):
                for g in grid:
                    if g == best[f]:
                        continue
                    trial = list(best)
                    trial[f] = g
                    t = score(trial)
                    if t < best_s:
                        best, best_s = trial, t
        self.gamma = best
        return {"gamma": best, "heldout_first_residual_geomean": float(np.exp(best_s)),
                "heldout_first_residual_geomean_least_squares": float(np.exp(start_s)),
                "heldout_first_residual_geomean_base": float(np.exp(base_s)),
                "heldout_steps_used": len(steps)}

    def predict(self, ts: TimeSeries, calibrated: bool = True, i: int | None = None, gamma=None,
                online: bool = False):
        """Initial guess for step i + 1 (default: the next step) from the stored steps up to i: the
        base extrapolation plus the network's correction, scaled per field by gamma (default the
        calibrated one; calibrated=False: unscaled)."""
        torch = self.torch
        N = self.N
        i = len(ts.x_hist) - 1 if i is None else i
        xin = torch.empty(self.in_ch * N * N, dtype=torch.float32, device="cuda")
        self._pack(ts, i, xin)
        d = torch.empty(3 * N * N, dtype=torch.float32, device="cuda")
        self.net.forward(xin, d, 1, N)
        g = torch.empty(3 * N * N, dtype=torch.float64, device="cuda")
        if gamma is None:
            gamma = self.online_gamma() if online else (self.gamma if calibrated else [1.0, 1.0, 1.0])
        gm = gamma
        sc = [s * g for s, g in zip(self.out_scale, gm)]
        api.ibnet_apply_delta(N, ts.x_hist[i], d, sc, g, **self._hist(ts, i))
        return g

    def extrapolate(self, ts: TimeSeries, order: int = 1):
        """The baselines without the network: 2 x^n - x^{n-1} (order 1) or
        3 x^n - 3 x^{n-1} + x^{n-2} (order 2)."""
        torch = self.torch
        N = self.N
        i = len(ts.x_hist) - 1
        g = torch.empty(3 * N * N, dtype=torch.float64, device="cuda")
        extra = dict(x_prev2=ts.x_hist[i - 1], x_prev3=ts.x_hist[i - 2] if order == 2 else None)
        api.ibnet_apply_delta(N, ts.x_hist[i], None, self.out_scale, g, **extra)
        return g


class ChannelSeries:
    """The flow-past-a-fiber time series in its channel (Sec. 5.3), keeping every step's
    solution and spread fiber force on the device, with the same attributes as TimeSeries
    (x_hist, f_hist) so that LearnedGuess trains and predicts on it unchanged.

    Every step is solved by Newton's method (fiber_channel.FiberChannel) from a predicted
    solution: Newton starts from it and every Newton system's FGMRES starts from the current
    iterate; FGMRES stops at fgmres_rtol relative to the system's right-hand side and Newton at
    newton_rtol relative to the step's base right-hand side, references that do not depend on
    the prediction, so predictions are compared on equal terms."""

    def __init__(self, rec, cav: dict | None = None, fgmres_rtol: float = 1e-10, newton_rtol: float = 1e-9):
        import torch
        from .fiber_channel import FiberChannel
        self.torch = torch
        self.fc = FiberChannel(rec, cav, newton_rtol=newton_rtol, fgmres_rtol=fgmres_rtol, newton_ref="b")
        self.rec0 = rec
        self.N = rec.N
        self.n = 3 * rec.N * rec.N
        self.t = 0.0
        self.x_hist = [torch.zeros(self.n, dtype=torch.float64, device="cuda")]  # w^0: at rest
        self.f_hist = []
        self.X_hist = []   # markers X^n at the start of step n (host), for first_residual
        self.records = []

    def _spread_force(self):
        torch = self.torch
        N = self.N
        sysm = api.ib_setup(self.fc.rec)
        F = torch.empty(2 * self.rec0.M, dtype=torch.float64, device="cuda")
        api.ib_force(sysm, F)
        f = torch.empty(2 * N * N, dtype=torch.float64, device="cuda")
        api.ib_spread(sysm, F, f)
        sysm.close()
        return f

    def step(self, guesses=(("previous", None),)):
        """One time step solved from every (label, fn[, precision]) entry: fn(self) returns the
        predicted solution once this step's spread force is stored (None: the previous step's
        solution); precision (default: the series') of the stored patch inverses.  Every entry
        starts from the same X^n; the first one's result advances the series.  Returns
        [(label, {newton, fgmres, fgmres_total, seconds, r0, converged})]."""
        self.f_hist.append(self._spread_force())
        t_next = self.t + self.rec0.dt
        rec_n = self.fc.rec
        self.X_hist.append(rec_n.X)
        prec0 = self.fc.cav.get("precision", "fp64")
        out, main = [], None
        for entry in guesses:
            label, fn = entry[0], entry[1]
            self.fc.cav["precision"] = entry[2] if len(entry) > 2 else prec0
            self.fc.rec = rec_n
            g = self.x_hist[-1] if fn is None else fn(self)
            w, X, hist, infos, sec = self.fc.step(self.x_hist[-1], t_next, guess=g)
            its = [i["iters"] for i in infos]
            out.append((label, {"newton": len(hist) - 1, "fgmres": its, "fgmres_total": int(sum(its)),
                                "seconds": sec, "r0": float(hist[0]),
                                "converged": all(i["converged"] for i in infos)}))
            if main is None:
                main = (w, X)
        self.fc.cav["precision"] = prec0
        self.fc.rec = replace(rec_n, X=main[1])
        self.x_hist.append(main[0])
        self.t = t_next
        self.records.append(out)
        return out

    def first_residual(self, i: int, guess) -> float:
        """The first Newton residual of the stored step from x^i to x^{i+1} started at `guess`
        (a past step, re-evaluated without solving)."""
        rec = replace(self.fc.rec, X=self.X_hist[i])
        return self.fc.first_residual(self.x_hist[i], (i + 1) * self.rec0.dt, guess, rec=rec)
