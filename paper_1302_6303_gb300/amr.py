"""Dynamic AMR time integration (Sec. 5-6) over the C ABI.

Every `regrid_every` steps the refinement indicators are evaluated on the
current solution (nrd_tag), the tagged cells are clustered into a new
hierarchy (nrd_regrid_boxes), and when the boxes change the state and its
time history are moved to the new hierarchy by conservative linear
refinement (nrd_transfer).  Warm restart: the step that produced the current
solution is solved again on the new hierarchy from the transferred solution,
with the transferred history, and the first local error estimate after the
regrid is not used for step control (Sec. 5).  Step control is that of
`stepper.Integrator` (leapfrog predictor, Eq. bdf2le, EPS or PC.4.7).

Host bookkeeping only; every vector operation runs in libnrd.so.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import nrd
from .workloads import Hierarchy


@dataclass
class RegridPolicy:
    regrid_every: int = 5
    thr_c: float = float("inf")      # tau^c threshold (bit 0)
    thr_g: float = float("inf")      # tau^g threshold (bit 1)
    thr_r: float = float("inf")      # h |grad E| / E threshold (bit 2)
    tag_bits: int = 7
    buffer: int = 1
    efficiency: float = 0.7
    min_side: int = 4
    max_side: int = 32
    max_levels: int = 3
    max_boxes: int = 4096


@dataclass
class RegridEvent:
    step: int
    t: float
    ncells_old: int
    ncells_new: int
    nboxes: list
    fnorm_before: float               # residual norm of the transferred state
    fnorm_after: float
    newton: int
    krylov: int
    regrid_s: float = 0.0             # tags, clustering, new context, transfer (wall)
    resolve_s: float = 0.0            # the re-solve, including the new context's graph build


class DynamicAmr:
    """Adaptive-step BDF2 with dynamic regridding on a fixed base grid.

    material: callable Hierarchy -> float32 numpy array of z per cell
    (material is a function of position, re-evaluated on every hierarchy).
    """

    def __init__(self, hier: Hierarchy, material, params=None, policy: RegridPolicy | None = None,
                 eps_t=5e-3, controller=nrd.DT_PC47, eta_E=1e-5, eta_T=1e-3, dt_max=None,
                 dt_min=1e-12, device="cuda"):
        self.material = material
        self.params = params
        self.policy = policy or RegridPolicy()
        self.eps_t, self.controller = eps_t, controller
        self.eta_E, self.eta_T = eta_E, eta_T
        self.dt_max, self.dt_min = dt_max, dt_min
        self.device = device
        self.hier = None
        self.ctx = None
        self._install(hier)
        self.history = []
        self.events: list[RegridEvent] = []

    # ------------------------------------------------------------ hierarchy
    def _new_ctx(self, hier):
        ctx = nrd.Context(self.params) if self.params is not None else nrd.Context()
        ctx.set_hierarchy_from(hier)
        z = torch.as_tensor(np.ascontiguousarray(self.material(hier), dtype=np.float32),
                            device=self.device)
        ctx.set_material(z)
        return ctx

    def _install(self, hier):
        self.hier = hier
        self.ctx = self._new_ctx(hier)

    def _regrid(self, vecs):
        """Cluster the tags of vecs[0]; if the boxes change, move every vector
        of `vecs` (None entries kept) to the new hierarchy.  Returns the new
        vectors, or None when the hierarchy stays."""
        p = self.policy
        tags = self.ctx.tag(vecs[0], p.thr_c, p.thr_g, p.thr_r)
        levels = self.ctx.regrid_boxes(tags, p.tag_bits, p.buffer, p.efficiency, p.min_side,
                                       p.max_side, p.max_levels, p.max_boxes)
        cur = [[(tuple(lo), tuple(hi)) for lo, hi in lev] for lev in self.hier.levels]
        if levels == cur:
            return None
        newh = Hierarchy(n0=self.hier.n0, levels=levels, bc_type=list(self.hier.bc_type),
                         bc_R=list(self.hier.bc_R))
        new_ctx = self._new_ctx(newh)
        live = [v for v in vecs if v is not None]
        moved = self.ctx.transfer_to(new_ctx, torch.stack(live))
        out, q = [], 0
        for v in vecs:
            if v is None:
                out.append(None)
            else:
                out.append(moved[q].contiguous())
                q += 1
        self.ctx.close()
        self.ctx = new_ctx
        self.hier = newh
        return out

    # ------------------------------------------------------------ stepping
    def run(self, u0, dt0, nsteps=None, t_end=None):
        t = 0.0
        un = u0.clone()
        unm1 = None
        udot = None
        dt, dt_prev = dt0, None
        err_prev = None
        ignore = False
        last = None        # (u_n, u_{n-1}, dt, dt_prev) of the step just taken
        n = 0
        while (nsteps is None or n < nsteps) and (t_end is None or t < t_end * (1 - 1e-12)):
            ctx = self.ctx
            if t_end is not None:
                dt = min(dt, t_end - t)
            if unm1 is None or udot is None:
                u = un.clone()
                st = ctx.step(u, un, None, dt)
                err, dtp = None, 0.0
            else:
                up = ctx.predict(un, unm1, udot, dt, dt_prev)
                u = up.clone()
                st = ctx.step(u, un, unm1, dt, dt_prev)
                err = ctx.lte(u, up, dt / dt_prev, self.eta_E, self.eta_T)
                dtp = dt_prev
            if st["status"] != nrd.OK:
                raise RuntimeError("step %d did not converge (status %d)" % (n, st["status"]))
            last = (un, unm1, dt, dtp, st["fnorm0"])
            udot = ctx.time_derivative(u, un, unm1, dt, dtp)
            t += dt
            self.history.append(dict(step=n, t=t, dt=dt, err=err, newton=st["newton_its"],
                                     krylov=st["krylov_its"], ncells=ctx.N,
                                     nleaf=ctx.nleaf, nlevels=ctx.nlevels))
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
            # ------------------------------------------------------ regrid
            if self.policy.regrid_every > 0 and n % self.policy.regrid_every == 0:
                h_un, h_unm1, h_dt, h_dtp, h_f0 = last
                old_ncells = self.ctx.N
                t_rg = time.perf_counter()
                moved = self._regrid([un, h_un, h_unm1])
                t_rg = time.perf_counter() - t_rg
                if moved is not None:
                    un_new, h_un_new, h_unm1_new = moved
                    ctx = self.ctx
                    # warm restart: re-solve the step on the new hierarchy from
                    # the transferred solution (Newton's first residual is the
                    # jump the transfer made).  It stops at the absolute
                    # residual the original step reached, rtol ||F(u^0)||:
                    # where the hierarchy changed only in smooth regions the
                    # transferred state is already converged and a purely
                    # relative test would ask for rounding noise.
                    u = un_new.clone()
                    t_rs = time.perf_counter()
                    atol0 = ctx.params.atol
                    ctx.set_params(atol=max(atol0, ctx.params.rtol * h_f0))
                    try:
                        st = ctx.step(u, h_un_new, h_unm1_new, h_dt, h_dtp, check=False)
                    finally:
                        ctx.set_params(atol=atol0)
                    t_rs = time.perf_counter() - t_rs
                    if st["status"] != nrd.OK:
                        raise RuntimeError("re-solve after regrid did not converge")
                    un, unm1 = u, h_un_new
                    udot = ctx.time_derivative(un, h_un_new, h_unm1_new, h_dt, h_dtp)
                    ignore = True
                    self.events.append(RegridEvent(
                        step=n, t=t, ncells_old=old_ncells, ncells_new=ctx.N,
                        nboxes=[len(l) for l in self.hier.levels], fnorm_before=st["fnorm0"],
                        fnorm_after=st["fnorm"], newton=st["newton_its"],
                        krylov=st["krylov_its"], regrid_s=t_rg, resolve_s=t_rs))
        return un
