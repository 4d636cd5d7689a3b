"""Gradients through implicit backward-Euler steps (differentiation pattern).

`ImplicitSteps` is a torch.autograd.Function around the C ABI: its forward
takes `nsteps` backward-Euler steps (nrd_step) from E0 with the material z and
returns the functional J = sum over the leaf cells of a box of V_c E_c at the
final time; its backward runs the discrete adjoint (nrd_linearise,
nrd_adjoint_solve, nrd_vjp) backwards through the steps, recomputing the
states of each segment from checkpoints stored every `ckpt_every` steps.

For one step F(u_{n+1}; u_n, z) = u_{n+1} - u_n - dt f(u_{n+1}; z) = 0:
  lam_n solves (dF/du_{n+1})^T lam_n = g_{n+1},
  g_n = -(dF/du_n)^T lam_n = lam_n,            dJ/dz -= (dF/dz)^T lam_n.
Only marshalling and the checkpoint schedule live here; every step of the
computation runs in libnrd.so.
"""
from __future__ import annotations

import torch


class StepRunner:
    """Holds the context and the fixed parts of the problem (T0, dt, steps)."""

    def __init__(self, ctx, T0, nsteps, dt, weights, ckpt_every=8, adjoint_rtol=1e-10):
        self.ctx = ctx
        self.T0 = T0
        self.nsteps = nsteps
        self.dt = dt
        self.weights = weights          # (N,) float64: V_c on leaf cells of the box, else 0
        self.ckpt_every = ckpt_every
        self.adjoint_rtol = adjoint_rtol
        self.stats = []           # nrd_step stats of every forward step (recomputations too)
        self.adjoint_stats = []   # nrd_adjoint_solve stats, one per step of the backward pass

    def step(self, un):
        u = un.clone()
        st = self.ctx.step(u, un, None, self.dt)
        self.stats.append(st)
        return u

    def run(self, u0, n):
        u = u0
        for _ in range(n):
            u = self.step(u)
        return u


class ImplicitSteps(torch.autograd.Function):
    @staticmethod
    def forward(actx, z, E0, runner: StepRunner):
        ctx = runner.ctx
        ctx.set_material(z.to(torch.float32).contiguous())
        N = E0.numel()
        u = torch.cat([E0, runner.T0]).contiguous()
        ckpts = []
        for n in range(runner.nsteps):
            if n % runner.ckpt_every == 0:
                ckpts.append(u.clone())
            u = runner.step(u)
        J = torch.dot(runner.weights, u[:N])
        actx.runner = runner
        actx.ckpts = ckpts
        actx.N = N
        return J

    @staticmethod
    def backward(actx, gJ):
        r = actx.runner
        ctx = r.ctx
        N = actx.N
        g = torch.zeros(2 * N, dtype=torch.float64, device=gJ.device)
        g[:N] = gJ * r.weights
        dz = torch.zeros(N, dtype=torch.float64, device=gJ.device)
        nseg = len(actx.ckpts)
        for sgi in reversed(range(nseg)):
            n0 = sgi * r.ckpt_every
            n1 = min(n0 + r.ckpt_every, r.nsteps)
            # recompute the states of this segment from its checkpoint
            states = [actx.ckpts[sgi]]
            for _ in range(n0, n1):
                states.append(r.step(states[-1]))
            for n in reversed(range(n0, n1)):
                un, unp1 = states[n - n0], states[n - n0 + 1]
                ctx.linearise(unp1, un, 1.0, r.dt)
                lam, ast = ctx.adjoint_solve(g, 1.0, r.dt, rtol=r.adjoint_rtol)
                r.adjoint_stats.append(ast)
                _, dzn = ctx.vjp(lam, 1.0, r.dt)
                dz -= dzn
                g = lam
        return dz, g[:N].clone(), None


def box_weights(hier, box):
    """V_c for leaf cells whose centre lies in `box` (base-cell units,
    inclusive lo/hi), else 0."""
    import numpy as np
    leaf = ~hier.covered_mask()
    L, x, y, z = hier.cell_centres()
    lo = np.array(box[0], dtype=np.float64)
    hi = np.array(box[1], dtype=np.float64) + 1.0
    nb = np.array(hier.n0, dtype=np.float64)
    inside = np.ones(x.size, dtype=bool)
    for d, c in enumerate((x, y, z)):
        inside &= (c * nb[d] >= lo[d]) & (c * nb[d] < hi[d])
    vol = np.array([1.0 / np.prod(hier.level_n(l)) for l in range(hier.nlevels)])[L]
    return np.where(inside & leaf, vol, 0.0)
