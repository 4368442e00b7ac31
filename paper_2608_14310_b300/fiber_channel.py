"""Time loop of the flow-past-a-fiber benchmark (Sec. 5.3) on the channel.

Each semi-implicit step t^n -> t^{n+1} is solved by Newton's method on (u, p), with the
fiber's force taken at the updated configuration X_k = X^n + dt J^n u_k (Eqs. im_disc_mom,
im_disc_advec): every Newton system K_E(X_k) w = rhs_k is solved by CAV-preconditioned FGMRES
with the hierarchy rebuilt for that system, as the paper does, starting from the iterate w_k
(its initial residual rhs_k - K_E(X_k) w_k is the Newton residual at w_k), so the FGMRES
tolerance is an inexact-Newton forcing term.  Host control flow only:
every arithmetic step (right-hand sides, force, E_E assembly, set-up, solves, residual
norms, marker advection) is a call of the C ABI in `api`.
"""
from __future__ import annotations

import math
import time
from dataclasses import replace

from . import api


def inflow_speed(t: float, U: float = 1.0, T_ramp: float = 0.5625) -> float:
    """The inflow speed at time t, raised smoothly from 0 to U over [0, T_ramp] (Sec. 5.3 says
    only "smoothly"; the ramp is the half cosine U (1 - cos(pi t / T)) / 2)."""
    if t >= T_ramp:
        return U
    return U * 0.5 * (1.0 - math.cos(math.pi * t / T_ramp))


DEFAULT_CAV = dict(kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, smoother="coloured", precision="fp64")


class FiberChannel:
    """Steps of the fiber in its channel from a record with bc = "channel" (ib_workloads)."""

    def __init__(self, rec, cav: dict | None = None, newton_rtol: float = 1e-8, newton_atol: float = 1e-8,
                 fgmres_rtol: float = 1e-9, newton_maxit: int = 20, fgmres_maxit: int = 150,
                 newton_ref: str = "r0", refactor: bool = True):
        """newton_ref "r0": stop when ||R(w_k)|| <= max(newton_rtol ||R(w_0)||, newton_atol) (the
        paper's relative test, as in the oracle); "b": ||R(w_k)|| <= newton_rtol ||b|| with b the
        step's base right-hand side, a reference independent of the starting iterate (used
        when comparing initial guesses).  refactor: a hierarchy is kept between Newton
        systems (and steps) and rebuilt numerically by cav_refactor while E_E's pattern is
        unchanged (bit for bit the hierarchy cav_setup would build), else by cav_setup."""
        assert getattr(rec, "bc", "periodic") == "channel"
        assert newton_ref in ("r0", "b")
        self.rec = rec
        self.cav = dict(DEFAULT_CAV if cav is None else cav)
        self.newton_rtol, self.newton_atol, self.newton_ref = newton_rtol, newton_atol, newton_ref
        self.fgmres_rtol, self.newton_maxit, self.fgmres_maxit = fgmres_rtol, newton_maxit, fgmres_maxit
        self.refactor = refactor
        self._h = {}          # hierarchies kept for refactorisation, by set-up parameters
        self.setups = 0       # cav_setup calls
        self.refactors = 0    # cav_refactor calls that succeeded

    def _hierarchy(self, sysm):
        """The hierarchy for the system's current E_E (Sec. 5.3 rebuilds it per Newton system)."""
        if not self.refactor:
            self.setups += 1
            return api.cav_setup(sysm, **self.cav)
        key = tuple(sorted(self.cav.items()))
        h = self._h.get(key)
        if h is not None and api.cav_refactor(h, sysm):
            self.refactors += 1
            return h
        if h is not None:
            h.close()
        h = api.cav_setup(sysm, **self.cav)
        self._h[key] = h
        self.setups += 1
        return h


    def first_residual(self, w_n, t_next: float, guess, rec=None) -> float:
        """||R(w_0)|| of the step from w_n (markers at rec.X, default self.rec) with Newton started
        at `guess`: the first Newton residual step() would record, without solving."""
        import torch
        rec = self.rec if rec is None else rec
        sysm = api.ib_setup(rec)
        b = torch.empty_like(w_n)
        api.ib_channel_rhs(sysm, w_n, inflow_speed(t_next), inflow_speed(t_next - rec.dt), b)
        w = guess.clone()
        X_k = api.ib_advect(sysm, w)
        api.ib_update_structure(sysm, replace(rec, meta={**rec.meta, "X_lin": X_k}))
        rhs = torch.empty_like(w_n)
        r = torch.empty_like(w_n)
        api.ib_newton_rhs(sysm, b, w, rhs)
        out = api.ib_residual_norm(sysm, rhs, w, r)
        sysm.close()
        return out

    def step(self, w_n, t_next: float, guess=None):
        """One step from the device vector w_n (3 N^2, at t^n = t_next - dt) with the markers at
        self.rec.X = X^n.  guess (device, optional): a prediction of the step's solution, used as
        Newton's starting iterate (without it Newton starts from w_n, as in the paper and the
        oracle).  Every Newton system's FGMRES solve starts from the current iterate.  Returns
        (w, X_next, residual history, FGMRES infos, seconds) and moves self.rec to X^{n+1}."""
        import torch
        rec = self.rec
        dt = rec.dt
        t0 = time.perf_counter()
        sysm = api.ib_setup(rec)
        b = torch.empty_like(w_n)
        api.ib_channel_rhs(sysm, w_n, inflow_speed(t_next), inflow_speed(t_next - dt), b)
        w = (w_n if guess is None else guess).clone()
        rhs = torch.empty_like(w_n)
        r = torch.empty_like(w_n)
        X_k = api.ib_advect(sysm, w)
        if self.newton_ref == "b":
            ref = api.ib_residual_norm(sysm, b, torch.zeros_like(w_n), r)  # ||b - K 0|| = ||b||
        hist, its = [], []
        k = 0
        while True:
            api.ib_update_structure(sysm, replace(rec, meta={**rec.meta, "X_lin": X_k}))
            api.ib_newton_rhs(sysm, b, w, rhs)
            hist.append(api.ib_residual_norm(sysm, rhs, w, r))
            tol = max(self.newton_rtol * hist[0], self.newton_atol) if self.newton_ref == "r0" else \
                self.newton_rtol * ref
            if k >= self.newton_maxit or hist[-1] <= tol:
                break
            h = self._hierarchy(sysm)
            x = w.clone()
            # newton_ref "r0": fgmres_rtol relative to the Newton residual at w_k (inexact Newton);
            # "b": relative to ||rhs_k||, a reference independent of the starting iterate
            info = api.fgmres_solve(sysm, h, rhs, x, rtol=self.fgmres_rtol, maxit=self.fgmres_maxit,
                                    rel_to=1 if self.newton_ref == "r0" else 0, history=False)
            if not self.refactor:
                h.close()
            its.append(info)
            w = x
            X_k = api.ib_advect(sysm, w)
            k += 1
        torch.cuda.synchronize()
        self.rec = replace(rec, X=X_k)
        return w, X_k, hist, its, time.perf_counter() - t0
