"""Adaptive variable-step BDF2 integration (Sec. 3.3-3.5) over the C ABI.

Each step: the generalised leapfrog predictor (Eq. leapfrog, with the time
derivative from the left-hand side of Eq. bdf2) gives the initial guess, the
Newton solve of Eq. nonlinearsystem advances the state, the local error of
Eq. bdf2le in the scaled max norm feeds the EPS (Eq. odets) or PC.4.7 (Eq.
pc47) controller.  After a change of hierarchy the first error estimate is
not used (Sec. 5).  The first step is backward Euler.  Host bookkeeping only;
all vector work runs in libnrd.so.
"""
from __future__ import annotations

import torch

from . import nrd


class Integrator:
    def __init__(self, ctx, eps_t=5e-4, controller=nrd.DT_PC47, eta_E=1e-5, eta_T=1e-3,
                 dt_max=None, dt_min=1e-12):
        self.ctx = ctx
        self.eps_t = eps_t
        self.controller = controller
        self.eta_E, self.eta_T = eta_E, eta_T
        self.dt_max, self.dt_min = dt_max, dt_min
        self.history = []

    def run(self, u0, dt0, nsteps=None, t_end=None, skip_first_lte=False):
        ctx = self.ctx
        t = 0.0
        un = u0.clone()
        unm1 = None
        udot = None
        dt, dt_prev = dt0, None
        err_prev = None
        ignore = skip_first_lte
        n = 0
        while (nsteps is None or n < nsteps) and (t_end is None or t < t_end * (1 - 1e-12)):
            if t_end is not None:
                dt = min(dt, t_end - t)
            if unm1 is None or udot is None:
                u = un.clone()
                st = ctx.step(u, un, None, dt)
                err = None
                alpha = 0.0
            else:
                up = ctx.predict(un, unm1, udot, dt, dt_prev)
                u = up.clone()
                st = ctx.step(u, un, unm1, dt, dt_prev)
                alpha = dt / dt_prev
                err = ctx.lte(u, up, alpha, self.eta_E, self.eta_T)
            # derivative at t_{n+1} from the left-hand side of the step just taken
            udot = ctx.time_derivative(u, un, unm1, dt, dt_prev if unm1 is not None else 0.0)
            t += dt
            rec = dict(step=n, t=t, dt=dt, err=err, newton=st["newton_its"],
                       krylov=st["krylov_its"], status=st["status"])
            self.history.append(rec)
            # next step size
            dt_next = dt
            if err is not None and err > 0.0 and not ignore:
                if self.controller == nrd.DT_PC47 and err_prev is not None:
                    dt_next = nrd.dt_control(nrd.DT_PC47, self.eps_t, err, err_prev, dt, dt_prev)
                else:
                    dt_next = nrd.dt_control(nrd.DT_EPS, self.eps_t, err, 0.0, dt, dt)
                err_prev = err
            elif err is not None:
                ignore = False
            if self.dt_max is not None:
                dt_next = min(dt_next, self.dt_max)
            dt_next = max(dt_next, self.dt_min)
            unm1, un = un, u
            dt_prev, dt = dt, dt_next
            n += 1
        return un
