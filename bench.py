#!/usr/bin/env python
"""Benchmark of the implicit radiation-diffusion hot path on one GB300.

Workloads (``--workload``; the default is the largest single-GPU one):

* ``single256`` (default): one level of 256^3 cells (16.8M) on the unit cube,
  z in {1, 5, 10} in 64 seeded cubes of side 8-32 cells, E0 = 1e-5,
  T0 = E0^(1/4), Robin R = 1 at x = 0, Neumann elsewhere.  FP64 Newton
  residual, Jv and FGMRES(30) orthogonalisation; FP32 4-level V-cycle with
  3 red-black Gauss-Seidel sweeps before and after; Newton rtol 1e-8.
* ``amr2_base64``: 2-level AMR, base 64^3, refinement ratio 2, fine patches
  of 16^3-32^3 cells tiling the Marshak band x < 1/8, z = 10 in 20 seeded
  cubes of side 4-12 base cells on z = 1; sweep schedule from the autotuner.
* ``batching_base128``: 3 levels, base 128^3, 1,913 patches with even sides
  uniform in 8-48 cells per axis (45.6M cells), z = 10 in 64 seeded cubes;
  sweep schedule from the autotuner; dt = 1e-4.

All: BDF2 steps (the first one backward Euler) with a fixed dt (5e-4 unless
stated) from the initial state (Sec. 3.1), Newton rtol 1e-8.

One benchmark step = one implicit time step through the public API: the
generalised leapfrog predictor as the Newton initial guess (nrd_predict, Eq.
leapfrog), the Newton solve (nrd_step: ghost fill, residual, Jv, GMRES,
preconditioner set-up and V-cycles, P2, Newton updates), the time derivative
at the new level for the next prediction (nrd_time_derivative), and the
refinement indicators (nrd_tag).

metric: Mcell/s of Jv + V-cycle = leaf cells x Krylov iterations (each one Jv
plus one P^{-1} application) / total implicit-step time.  Reported for the
production form (analytic Jv, FP32 V-cycle) with the plain form (FD Jv, FP64
V-cycle) measured on the same workload beside it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM, FALLBACK_BF16 = 6800.0, 1900.0
DT = 5e-4   # the time step of the selected workload (set from WORKLOADS in main)

# The workloads.  `solver` holds the V-cycle schedule where the workload
# states one (three red-black Gauss-Seidel sweeps: V(3,3) with 2 x 3 sweeps on
# the coarsest grid); None lets the sweep autotuner choose.  `cpu_n` is the
# grid of the bounded oracle sample timed on the host (the same layout
# scaled), None for the full workload.  `dt`: the fixed time step.  `tile`: the
# stencil tile the autotuner picks for the workload in the recorded runs (used
# by the profiling modes, which skip the autotuner).
WORKLOADS = {
    "single256": {
        "name": "single_level_256cubed_64cubes_z1_5_10",
        "sizes": "256^3 cells, one level",
        "solver": dict(nmg=4, nu1=3, nu2=3, coarse_sweeps=6),
        "regrid": False,
        "cpu_n": 128,
        "dt": 5e-4,
        "tile": (8, 8, 8),
    },
    "amr2_base64": {
        "name": "amr2_base64_marshak_band",
        "sizes": "base 64^3 + 31 fine patches of 16^3-32^3 cells",
        "solver": None,
        "regrid": True,
        "cpu_n": None,
        "dt": 5e-4,
        "tile": (8, 8, 4),
    },
    "batching_base128": {
        "name": "batching_base128_3levels",
        "sizes": "base 128^3 + two levels of patches with sides 8-48 per axis (about 1,900 "
                 "patches, 45.6M fine cells), fixed hierarchy",
        "solver": None,
        "regrid": False,
        "cpu_n": 32,
        # finest cells 1/512 wide: from the cold start, dt = 5e-4 takes Newton
        # past 20 iterations on the first step (4 at dt = 1e-4)
        "dt": 1e-4,
        "tile": (8, 8, 4),
    },
}

# Algorithmic FP64 work per leaf cell, counted from the formulas of Sec. 3.2
# and Sec. 4.2 (each add, subtract or multiply one operation; divisions and
# square roots charged below at their measured cost):
#  residual, per face (3 per cell): T_f 2, z_a^3 + z_b^3 1, 3(...) 1, T_f^3 2,
#    E_a + E_b 1, its scaling 1, dE 1, 2 D_r 1, D_h g 1, 1 + D_h g 1,
#    k T_f^2 sqrt(T_f) 2, the two fluxes 2 + 2 with dT 1: 19 ops, 3 divisions
#    (D_r, g, D_E), 1 square root; per cell: z^3 2, the two divergences 16,
#    T^3 2, T^4 1, T^4 - E 1, sigma (T^4 - E) 1, a0 u - b - dt (div +- coupling)
#    5 + 5: 33 ops, 1 division (sigma): 90 ops, 10 divisions, 3 square roots.
#  linearisation = residual + per face the five flux partials (dD_r/dT_f 1,
#    dg/dE_a, dg/dE_b 5, dD_E/dD_h and dD_E/dg 2, the chain to T_f 2 and to
#    E_a, E_b 2, dF_E 3 + 3 + 2, dD_T/dT_f 2, dF_T 3 + 3) and the two scaled
#    P1 coefficients 2: 31 ops and 2 divisions (1/T_f, 1/(E_a + E_b)); per
#    cell the coupling partials 7 ops and 1 division, the P2 data 4 ops and
#    1 division: 194 ops, 18 divisions, 3 square roots.
#  frozen Jv: per face 6 + 3 (the two tangent fluxes from the five partials),
#    per cell the two divergences 16, the coupling tangent 3, a0 v - dt (...)
#    6: 52 ops.
LIN_OPS = (194, 18, 3)            # (ops, divisions, square roots) per leaf cell
RES_OPS = (90, 10, 3)
JV_OPS = (52, 0, 0)
# frozen-Jacobian Jv: 3 faces x 5 partials x 8 B + v 16 B + cell partials
# 16 B + Jv 16 B + mask 1 B
JV_BYTES_PER_CELL = 169.0
# DRAM bytes per launch group from an ncu capture of the current kernels,
# per workload (None: not captured for this kernel version and workload)
# (single256: captured on the same layout at 128^3, 2,097,152 cells, and
# scaled by the cells, x8: these stencils stream their inputs once; the
# linearisation's face and cell launches 58.1 + 394.5 + 187.8 + 64.9 MB,
# the frozen Jv 322.0 + 55.6 MB)
TRAFFIC = {
    "amr2_base64": {"linearise": None, "jv": None},
    "batching_base128": {"linearise": None, "jv": None},
    "single256": {"linearise": 8 * (58.1 + 394.5 + 187.8 + 64.9) * 1e6,
                  "jv": 8 * (322.0 + 55.6) * 1e6},
}
# FP64-pipe instructions per cell measured by ncu (sm__inst_executed_pipe_fp64,
# same capture): linearisation 139.2 + 35.0, frozen Jv 40.4
LIN_INST_NCU, JV_INST_NCU = 139.2 + 35.0, 40.4
# Algorithmic DRAM bytes per leaf cell of the linearisation as laid out here:
# face launch reads E, T, z^3 (24 B) and writes per face slot (3 per cell) the
# 5 FP64 Jacobian partials, the 2 scaled FP32 P1 coefficients and the 2 FP64
# face fluxes (3 x 64 = 192 B); the cell launch reads the 6 fluxes of its
# low faces (48 B), u and b (32 B) and z^3 (8 B) and writes F (16 B), the 2
# FP64 coupling partials (16 B) and the 3 FP32 P2 values (12 B).  The residual
# alone moves 52 B per cell and the analytic Jv 52 B (E, T, v, z read, Jv
# written); the frozen form stores the partials once per Newton iterate so
# that each Krylov iteration reads them instead of recomputing them in FP64.
# (ncu's DRAM bytes of a launch can fall below these counts: writes still held
# in the 129 MB L2 when the launch ends are counted by a later one.)
LIN_BYTES_PER_CELL = 24 + 192 + 48 + 32 + 8 + 16 + 16 + 12
RES_BYTES_PER_CELL = 52.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="single256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-regrid", action="store_true", help="skip the regrid/transfer leg")
    ap.add_argument("--profile", action="store_true",
                    help="short run for profilers: 1 warm-up + 2 production steps, fixed "
                         "8x8x4 tiles, the workload's sweep schedule (V(1,1)/2 where the "
                         "autotuner would choose), no plain/CPU/e2e legs; the "
                         "Newton loop runs host-driven so that a profiler sees every kernel "
                         "as its own launch (--profile-graph keeps the graph form)")
    ap.add_argument("--profile-graph", action="store_true")
    ap.add_argument("--profile-stencils", action="store_true",
                    help="short run for profilers: two rounds of linearisation, frozen Jv and "
                         "residual, then one Newton step (graph form), 8x8x8 tiles, GMRES "
                         "restart 2")
    ap.add_argument("--grid", type=int, default=0, metavar="N",
                    help="profile modes: the workload's layout at base N^3 (a smaller case of "
                         "the same kernels for multi-pass profiler captures)")
    ap.add_argument("--levels-table", type=float, default=0.0, metavar="T_END",
                    help="iteration table of Sec. 6: the dynamic-AMR Marshak run at base 16^3 "
                         "with at most 2, 3 and 4 levels to t = T_END (the paper's solver "
                         "settings); prints one JSON line per depth and exits")
    ap.add_argument("--profile-pc", type=int, default=0, metavar="N",
                    help="short run for profilers: N preconditioner applies (cached graph) "
                         "on the workload after one set-up, 8x8x4 tiles, the workload's "
                         "schedule (else V(1,1)/2); prints the mean time per apply")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the differentiation workload instead: base 96^3 + 8 fine boxes, "
                         "40 backward-Euler steps with checkpoints every 8, the gradient of "
                         "the final-time energy in a box with respect to z and E_0")
    ap.add_argument("--pc-sweeps", default="", metavar="NU1,NU2,COARSE,SMOOTHER",
                    help="V-cycle schedule of --profile-pc (smoother 0 red-black, 1 Jacobi, "
                         "2 x-line); default: the workload's, else V(1,1) red-black, 2 coarse")
    return ap.parse_args()


def profile_run(args):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd
    h, z, u0 = workload(args.workload)
    ctx = make_ctx(nrd, h, z, torch, production=True, wl=WORKLOADS[args.workload])
    tx, ty, tz = WORKLOADS[args.workload]["tile"]
    ctx.set_params(tile_x=tx, tile_y=ty, tile_z=tz, graph=1 if args.profile_graph else 0)
    if WORKLOADS[args.workload]["solver"] is None:
        ctx.set_params(nu1=1, nu2=1, coarse_sweeps=2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    r = run_steps(ctx, torch, u0, 2, 1, flush, timing=False)
    print(json.dumps({"profile_run": True, "ms": r["ms"], "krylov": r["krylov"]}))
    return 0


def profile_pc_run(args):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd
    h, z, u0 = workload(args.workload, args.grid or None)
    ctx = make_ctx(nrd, h, z, torch, production=True, wl=WORKLOADS[args.workload])
    ctx.set_params(tile_x=8, tile_y=8, tile_z=4)
    if args.pc_sweeps:
        n1, n2, cs, sm = (int(x) for x in args.pc_sweeps.split(","))
        ctx.set_params(nu1=n1, nu2=n2, coarse_sweeps=cs, smoother=sm)
    elif WORKLOADS[args.workload]["solver"] is None:
        ctx.set_params(nu1=1, nu2=1, coarse_sweeps=2)
    u = torch.from_numpy(u0).cuda()
    ctx.precond_setup(u, 1.0, DT)
    w = torch.from_numpy(np.random.default_rng(5).standard_normal(u0.size)).cuda()
    y = torch.empty_like(w)
    ctx.precond_apply(w, out=y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.profile_pc):
        ctx.precond_apply(w, out=y)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_pc": True, "applies": args.profile_pc, "cells": h.ncells,
                      "us_per_apply": e0.elapsed_time(e1) * 1e3 / args.profile_pc}))
    return 0


def adjoint_run(args):
    """The differentiation workload (Sec. 6 geometry): forward = 40 backward-
    Euler steps through ImplicitSteps (nrd_step, checkpoints every 8 steps),
    backward = the discrete adjoint through the steps (per step nrd_linearise,
    nrd_adjoint_solve with P^-T ~ P1^-1 P2^-T, nrd_vjp; each segment's states
    recomputed from its checkpoint), both timed with CUDA events; forward
    Newton rtol 1e-10, adjoint rtol 1e-10, analytic Jv, FP32 V-cycle."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd, workloads as W
    from paper_1302_6303_gb300.adjoint import ImplicitSteps, StepRunner, box_weights
    n0, nsteps, dt, ckpt = 96, 40, 2.5e-4, 8
    h, z, fbox = W.config_adjoint(n0, seed=0, nbox=8)
    u0 = W.front_state(h, seed=2, noise=0.0, front=0.5, width=0.05)
    N = h.ncells
    nmg = 1
    while nmg < 4 and all(n % (1 << nmg) == 0 for n in h.n0):
        nmg += 1
    ctx = nrd.Context(nmg=nmg, jv_mode=nrd.JV_ANALYTIC, pc_precision=nrd.PC_F32, rtol=1e-10,
                      atol=0.0, max_newton=30)
    ctx.set_hierarchy_from(h)
    ctx.set_material(torch.from_numpy(z).cuda())
    wts = torch.from_numpy(box_weights(h, fbox)).cuda()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    res = []
    for rep in range(1 + max(1, args.steps // 10)):
        runner = StepRunner(ctx, dev(u0[N:]), nsteps, dt, wts, ckpt_every=ckpt)
        zt = dev(z.astype(np.float64)).requires_grad_(True)
        Et = dev(u0[:N]).requires_grad_(True)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record()
        J = ImplicitSteps.apply(zt, Et, runner)
        e1.record()
        nfwd = len(runner.stats)
        J.backward()
        e2.record()
        torch.cuda.synchronize()
        fst, bst, ast = runner.stats[:nfwd], runner.stats[nfwd:], runner.adjoint_stats
        res.append({"forward_ms": e0.elapsed_time(e1), "backward_ms": e1.elapsed_time(e2),
                    "forward_newton": sum(s["newton_its"] for s in fst),
                    "forward_krylov": sum(s["krylov_its"] for s in fst),
                    "recomputed_steps": len(bst),
                    "recompute_krylov": sum(s["krylov_its"] for s in bst),
                    "adjoint_krylov": sum(s["krylov_its"] for s in ast),
                    "J": float(J.detach())})
    r = res[-1]   # the first repetition also builds the graphs
    leaf = ctx.nleaf
    print(json.dumps({
        "adjoint": True, "workload": "differentiation: base 96^3 + 8 fine boxes of 16-32 fine "
        "cells near x = 0, 40 backward-Euler steps of dt = 2.5e-4, checkpoints every 8, "
        "J = integral of E over the interior (n0/6)^3 box at the final time",
        "cells": N, "leaf_cells": leaf, "repetitions": len(res), "timed": "the last one",
        "forward_ms": r["forward_ms"], "backward_ms": r["backward_ms"],
        "backward_over_forward": r["backward_ms"] / r["forward_ms"],
        "forward_ms_per_step": r["forward_ms"] / nsteps,
        "forward_newton_per_step": r["forward_newton"] / nsteps,
        "forward_krylov_per_step": r["forward_krylov"] / nsteps,
        "recomputed_steps": r["recomputed_steps"],
        "adjoint_krylov_per_step": r["adjoint_krylov"] / nsteps,
        "forward_mcells": leaf * r["forward_krylov"] / (r["forward_ms"] * 1e-3) / 1e6,
        "gradient": "dJ/dz on the leaf cells and dJ/dE_0, checked against central differences "
                    "and the oracle's gradient in tests/test_gpu_adjoint.py",
        "J": r["J"], "all": res}))
    return 0


def profile_stencils_run(args):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd, workloads as W
    h, z, u0 = workload(args.workload, args.grid or None)
    sv = dict(nu1=2, nu2=2, nmg=4, coarse_sweeps=4)
    sv.update(WORKLOADS[args.workload]["solver"] or {})
    ctx = nrd.Context(restart=2, rtol=1e-8, jv_mode=nrd.JV_ANALYTIC, pc_precision=nrd.PC_F32,
                      tile_x=8, tile_y=8, tile_z=8, **sv)
    ctx.set_hierarchy_from(h)
    ctx.set_material(torch.from_numpy(z).cuda())
    u = torch.from_numpy(W.front_state(h, seed=1, noise=0.0, front=0.1, width=0.05)).cuda()
    v = torch.from_numpy(W.random_direction(h, 2)).cuda()
    for _ in range(2):
        ctx.linearise(u, u, 1.0, DT)
        ctx.jv(u, v, 1.0, DT, mode=nrd.JV_FROZEN)
        ctx.residual(u, u, 1.0, DT)
    un = u.clone()
    st = ctx.step(u, un, None, DT)
    torch.cuda.synchronize()
    print(json.dumps({"profile_stencils": True, "cells": h.ncells, "newton": st["newton_its"],
                      "krylov": st["krylov_its"]}))
    return 0


def levels_table(args):
    """Average Newton and GMRES iterations per time step of the dynamic-AMR
    Marshak run (Sec. 6: three z = 10 blocks, Robin R = 1 at x = 0 and R = 0
    at x = 1, E0 = 1e-5) at base 16^3 with at most 2, 3 and 4 levels, BDF2
    with the PC.4.7 controller, regridding every 4 steps on the tau^c and
    tau^g indicators, Newton rtol 1e-12 and atol 1e-10, at most 50 Krylov
    iterations per Newton step, V(1,0) red-black Gauss-Seidel with smoothing
    only on the coarsest level, FP32 V-cycle, analytic Jv."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd, workloads as W
    from paper_1302_6303_gb300.amr import DynamicAmr, RegridPolicy
    n0 = (16, 16, 16)
    cubes = W.paper_blocks(n0)
    h = W.Hierarchy(n0=n0, levels=[[((0, 0, 0), (15, 15, 15))]], bc_type=[1, 1, 0, 0, 0, 0],
                    bc_R=[1.0, 0.0, 0, 0, 0, 0])
    # the paper's 16b2l .. 16b4l averages (Sec. 6 iteration tables)
    paper = {2: (2.99, 7.71), 3: (2.96, 7.21), 4: (2.64, 6.63)}
    for L in (2, 3, 4):
        params = nrd.default_params(nu1=1, nu2=0, nmg=1, coarse_sweeps=1, rtol=1e-12, atol=1e-10,
                                    max_krylov=50, jv_mode=nrd.JV_ANALYTIC,
                                    pc_precision=nrd.PC_F32)
        pol = RegridPolicy(regrid_every=4, thr_c=0.2, thr_g=0.2, tag_bits=3, buffer=1,
                           efficiency=0.7, min_side=4, max_side=16, max_levels=L)
        run = DynamicAmr(h, lambda hh: W.material_from_cubes(hh, cubes), params=params,
                         policy=pol, eps_t=5e-3, dt_max=5e-3)
        t0 = time.perf_counter()
        run.run(torch.from_numpy(W.initial_state(h)).cuda(), 1e-4, t_end=args.levels_table)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        hist = run.history
        ns = len(hist)
        print(json.dumps({
            "levels": L, "t_end": args.levels_table, "steps": ns,
            "newton_per_step": sum(r["newton"] for r in hist) / ns,
            "gmres_per_step": sum(r["krylov"] for r in hist) / ns,
            "regrids": len(run.events), "max_leaf_cells": max(r["nleaf"] for r in hist),
            "levels_reached": max(r["nlevels"] for r in hist), "wall_s": wall,
            "regrid_s": sum(e.regrid_s for e in run.events),
            "resolve_s": sum(e.resolve_s for e in run.events),
            "paper_16b%dl" % L: {"newton_per_step": paper[L][0], "gmres_per_step": paper[L][1],
                                 "t_end": 1.0}}), flush=True)
    return 0


def replicas_value(dist, world, units, ms, device):
    """Whole-job rate of `world` replicas in Mcell/s: every rank processed
    `units` cell-iterations in `ms` of its own time; the job took the slowest
    rank's time (max over ranks).  Returns (rate, max ms)."""
    if dist is not None:
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units / (ms * 1e-3) / 1e6, ms


def workload(key, n=None):
    """Hierarchy, material and initial state of workload `key` (`n`: the
    base grid of a scaled copy, for the host sample)."""
    from paper_1302_6303_gb300 import workloads as W
    if key == "single256":
        h, z = W.config_256(n or 256, seed=0)
    elif key == "batching_base128":
        h, z = W.config_batching(n or 128, seed=0)
    else:
        h, z = W.config_amr2(n or 64, seed=0)
    return h, z, W.initial_state(h)


def peaks():
    if os.path.exists(MEASURED):
        d = json.load(open(MEASURED))
        return float(d.get("hbm_gbs", FALLBACK_HBM)), "measured"
    return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_ctx(nrd, h, z, torch, production, wl=None):
    if production:
        p = dict(jv_mode=nrd.JV_ANALYTIC, pc_precision=nrd.PC_F32)
    else:
        p = dict(jv_mode=nrd.JV_FD, pc_precision=nrd.PC_F64)
    sv = dict(nu1=2, nu2=2, nmg=4, coarse_sweeps=4)
    if wl is not None and wl["solver"] is not None:
        sv.update(wl["solver"])
    ctx = nrd.Context(restart=30, rtol=1e-8, **sv, **p)
    ctx.set_hierarchy_from(h)
    ctx.set_material(torch.from_numpy(z).cuda())
    return ctx


def run_steps(ctx, torch, u0, nsteps, warmup, flush, timing=False):
    """Integrate warmup + nsteps BDF2 steps (first BE); time the last nsteps
    with CUDA events per step (L2 flushed between steps, outside the events).
    A step is the paper's: the generalised leapfrog predictor (Eq. leapfrog,
    with the time derivative from the left-hand side of the previous step)
    gives the Newton initial guess, the Newton solve, the time derivative at
    the new level, the refinement indicators."""
    dev = torch.device("cuda")
    un = torch.from_numpy(u0).to(dev)
    unm1 = None
    udot = None
    u = un.clone()
    ud_next = torch.empty_like(un)
    tags = None
    times, kry, newt, kern = [], 0, 0, 0
    for s in range(warmup + nsteps):
        timed = s >= warmup
        if timed and s == warmup:
            torch.cuda.synchronize()
            if timing:
                ctx.timing_enable(True)
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        if udot is None:
            u.copy_(un)
        ev0.record()
        if udot is not None:
            ctx.predict(un, unm1, udot, DT, DT, out=u)
        # the time derivative and the indicators are enqueued behind the
        # Newton solve before the host waits for it (no idle gap)
        ctx.step_begin(u, un, unm1, DT, DT if unm1 is not None else 0.0)
        ctx.time_derivative(u, un, unm1, DT, DT if unm1 is not None else 0.0, out=ud_next)
        tags = ctx.tag(u, thr_r=0.1)
        ev1.record()
        st = ctx.step_end()
        torch.cuda.synchronize()
        if timed:
            times.append(ev0.elapsed_time(ev1))
            kry += st["krylov_its"]
            newt += st["newton_its"]
            kern += st["kernels"]
        unm1 = un
        un = u
        u = torch.empty_like(un)
        udot, ud_next = ud_next, (udot if udot is not None else torch.empty_like(un))
    kt = ctx.timing_read() if timing else None
    if timing:
        ctx.timing_enable(False)
    return dict(ms=times, krylov=kry, newton=newt, kernel=kt, u=un, u_prev=unm1, tags=tags,
                kernels=kern)


def run_e2e(nrd, ctx, torch, u0, nsteps, warmup):
    """Same metric through the public API with host buffers: each step copies
    the state u_n from pinned host memory, predicts, steps, forms the new time
    derivative, tags, and reads u_{n+1} and the tags back.  The history the
    next step needs (u_{n-1}, the time derivative) is what the previous step
    left on the device, as a caller that keeps it there would."""
    N2 = u0.size
    # the host buffers are pinned and stay so: the next step's input is
    # copied into them on the host, outside the timed region (a clone of a
    # pinned tensor is pageable, which would make the upload a staged copy)
    hn = torch.from_numpy(u0.copy()).pin_memory()
    hout = torch.empty(N2, dtype=torch.float64).pin_memory()
    htag = torch.empty(N2 // 2, dtype=torch.uint8).pin_memory()
    d_n = torch.empty(N2, dtype=torch.float64, device="cuda")
    d_nm1 = torch.empty_like(d_n)
    d_dot = torch.empty_like(d_n)
    d_dot_new = torch.empty_like(d_n)
    d_u = torch.empty_like(d_n)
    have_nm1 = have_dot = False
    total, kry = 0.0, 0
    h2d = d2h = 0
    side = torch.cuda.Stream()
    stepped, copied = torch.cuda.Event(), torch.cuda.Event()
    for s in range(warmup + nsteps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        d_n.copy_(hn, non_blocking=True)
        if have_dot:
            ctx.predict(d_n, d_nm1, d_dot, DT, DT, out=d_u)
        else:
            d_u.copy_(d_n)
        nm1 = d_nm1 if have_nm1 else None
        ctx.step_begin(d_u, d_n, nm1, DT, DT if have_nm1 else 0.0)
        # u_{n+1} goes back to the host on a side stream while the time
        # derivative and the indicators run (both only read it)
        stepped.record()
        with torch.cuda.stream(side):
            side.wait_event(stepped)
            hout.copy_(d_u, non_blocking=True)
            copied.record()
        ctx.time_derivative(d_u, d_n, nm1, DT, DT if have_nm1 else 0.0, out=d_dot_new)
        t = ctx.tag(d_u, thr_r=0.1)
        htag.copy_(t, non_blocking=True)
        torch.cuda.current_stream().wait_event(copied)
        ev1.record()
        st = ctx.step_end()
        torch.cuda.synchronize()
        if s >= warmup:
            total += ev0.elapsed_time(ev1)
            kry += st["krylov_its"]
            h2d, d2h = N2 * 8, N2 * 8 + N2 // 2
        hn.copy_(hout)
        # device history for the next step: this step's input and derivative
        d_nm1, d_n = d_n, d_nm1
        d_dot, d_dot_new = d_dot_new, d_dot
        have_nm1 = have_dot = True
    return total, kry, h2d, d2h


def regrid_leg(nrd, ctx, torch, h, z, r):
    """One regrid of the benchmark state (Sec. 5), outside the timed steps:
    device tags, host Berger-Rigoutsos clustering, conservative transfer of
    u_n and u_{n-1} to the new hierarchy, and the warm-restart re-solve."""
    from paper_1302_6303_gb300 import workloads as W
    u = r["u"]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tags = ctx.tag(u, thr_r=0.1)
    e1.record()
    torch.cuda.synchronize()
    tag_ms = e0.elapsed_time(e1)
    t0 = time.perf_counter()
    levels = ctx.regrid_boxes(tags, tag_bits=4, buffer=1, efficiency=0.7, min_side=16,
                              max_side=32, max_levels=2)
    cluster_ms = (time.perf_counter() - t0) * 1e3
    nh = W.Hierarchy(n0=h.n0, levels=levels, bc_type=h.bc_type, bc_R=h.bc_R)
    _, cubes = W.config_amr2_cubes(h.n0[0], seed=0)
    cn = make_ctx(nrd, nh, W.material_from_cubes(nh, cubes), torch, production=True,
                  wl=WORKLOADS["amr2_base64"])
    cn.set_params(tile_x=ctx.params.tile_x, tile_y=ctx.params.tile_y, tile_z=ctx.params.tile_z,
                  nu1=ctx.params.nu1, nu2=ctx.params.nu2, coarse_sweeps=ctx.params.coarse_sweeps,
                  smoother=ctx.params.smoother)
    hist = torch.stack([u, r["u_prev"]])
    cn.timing_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    moved = ctx.transfer_to(cn, hist)
    transfer_ms = (time.perf_counter() - t0) * 1e3
    k_ms, _ = cn.timing_read()["transfer"]
    cn.timing_enable(False)
    No, Nn, nvec = ctx.N, cn.N, 2
    alg = 2 * 16 * nvec * No + 4 * Nn + 2 * 16 * nvec * Nn
    # warm restart: the last step solved again (backward-Euler form from the
    # transferred u_{n-1}) from the transferred u_n
    un = moved[0].contiguous()
    e0.record()
    st = cn.step(un, moved[1].contiguous(), None, DT)
    e1.record()
    torch.cuda.synchronize()
    return {"tag_ms": tag_ms, "cluster_ms_host": cluster_ms, "boxes": [len(l) for l in levels],
            "leaf_cells_new": cn.nleaf, "transfer_ms_total": transfer_ms,
            "transfer_kernel_ms": k_ms, "transfer_vectors": nvec,
            "transfer_gbs": alg / (k_ms * 1e-3) / 1e9 if k_ms > 0 else None,
            "transfer_bytes": "copy of the old vectors (read+write) + 4 B source code per new "
                              "cell + one read and one write per new value (the 44 B entries "
                              "of reconstructed cells not counted)",
            "resolve_ms": e0.elapsed_time(e1), "resolve_newton": st["newton_its"],
            "resolve_krylov": st["krylov_its"], "fnorm_after_transfer": st["fnorm0"],
            "fnorm_resolved": st["fnorm"]}


def host_cpu():
    """Host core count and CPU model (nproc, lscpu)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_krylov_rate(h, z, u0, sweeps, threads, budget_s, min_its=2):
    """The oracle as it stands, on `threads` host threads: preconditioner
    set-up, then Krylov iterations' worth of P^{-1} (FAC/GMG) and analytic Jv
    until `budget_s` seconds have passed (at least `min_its`), with the
    V-cycle schedule and smoother the GPU run uses (sweeps = (nu1, nu2,
    coarse sweeps, smoother)).  Returns (Mcell/s, iterations, seconds)."""
    from oracle.oracle import Oracle, JV_ANALYTIC, set_threads
    set_threads(threads)
    o = Oracle(h, z)
    o.set_solver(jv_mode=JV_ANALYTIC, nu1=int(sweeps[0]), nu2=int(sweeps[1]), nmg=4,
                 coarse_sweeps=int(sweeps[2]))
    if len(sweeps) > 3 and int(sweeps[3]) == 1:   # damped Jacobi
        o.set_smoother(1, 6.0 / 7.0)
    leaf = int(o.leaf_mask().sum())
    rng = np.random.default_rng(0)
    w = rng.standard_normal(u0.size)
    o.pc_setup(u0, 1.0, DT)
    its = 0
    t0 = time.perf_counter()
    while its < min_its or time.perf_counter() - t0 < budget_s:
        y = o.pc_apply(w)
        w = o.jv_analytic(u0, y, 1.0, DT)
        w /= np.sqrt(max(o.dot(w, w), 1e-300))
        its += 1
    dt = time.perf_counter() - t0
    return leaf * its / dt / 1e6, its, dt, leaf


def oracle_step_seconds(h, z, u0, sweeps, threads):
    """Seconds of one oracle implicit step (backward Euler from u0, the
    GPU schedule, analytic Jv, rtol 1e-8) on `threads` host threads."""
    from oracle.oracle import Oracle, JV_ANALYTIC, set_threads
    set_threads(threads)
    o = Oracle(h, z)
    o.set_solver(jv_mode=JV_ANALYTIC, nu1=int(sweeps[0]), nu2=int(sweeps[1]), nmg=4,
                 coarse_sweeps=int(sweeps[2]), rtol=1e-8)
    if len(sweeps) > 3 and int(sweeps[3]) == 1:
        o.set_smoother(1, 6.0 / 7.0)
    t0 = time.perf_counter()
    _, st = o.newton(u0.copy(), u0.copy(), 1.0, DT)
    return time.perf_counter() - t0, st


def cpu_baseline(key, sweeps):
    """The oracle timed on the host cores, single thread and all cores: Jv +
    V-cycle Mcell/s on a bounded sample of the workload (the full workload,
    or the same layout at a smaller grid), and the seconds of one implicit
    step on the 64^3 version of the layout."""
    from paper_1302_6303_gb300 import workloads as W  # noqa: F401
    wl = WORKLOADS[key]
    h, z, u0 = workload(key, wl["cpu_n"])
    cores, model = host_cpu()
    v1, it1, s1, leaf = oracle_krylov_rate(h, z, u0, sweeps, 1, 8.0)
    vn, itn, sn, _ = oracle_krylov_rate(h, z, u0, sweeps, cores, 8.0)
    hs, zs, us = workload(key, 64 if key == "single256" else 16)
    step_s, st = oracle_step_seconds(hs, zs, us, sweeps, cores)
    where = ("the full workload" if wl["cpu_n"] is None
             else "the %d^3 version of the layout" % wl["cpu_n"])
    return {"value": vn, "unit": "Mcell/s", "cores": cores, "kind": "oracle",
            "sample": "Krylov iterations (P^-1 FAC/GMG apply + analytic Jv) of the FP64 oracle "
                      "on %s (%d leaf cells): %d iterations in %.1f s on %d threads; "
                      "single thread %.3f Mcell/s (%d iterations in %.1f s)"
                      % (where, leaf, itn, sn, cores, v1, it1, s1),
            "single_thread": {"value": v1, "unit": "Mcell/s", "iterations": it1, "seconds": s1},
            "cpu_model": model, "nproc": cores,
            "step": {"seconds": step_s, "threads": cores,
                     "workload": "one backward-Euler step of the same layout at base %d^3 "
                                 "(%d cells) from the initial state"
                                 % (hs.n0[0], hs.ncells),
                     "newton_its": st["newton_its"], "krylov_its": st["krylov_its"]}}


def reference_arm(args):
    """The oracle timed as the reference arm: each step = one Krylov iteration
    (P^{-1} + Jv) of the oracle on all host cores, on the workload, or for
    the 256^3 workload on its 128^3 version (a bounded sample: the metric is
    per cell)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    key = args.workload
    wl = WORKLOADS[key]
    h, z, u0 = workload(key, wl["cpu_n"])
    from oracle.oracle import Oracle, JV_ANALYTIC, set_threads
    cores, model = host_cpu()
    set_threads(cores)
    o = Oracle(h, z)
    sv = wl["solver"] or dict(nu1=1, nu2=1, coarse_sweeps=2)
    # the GPU run's V-cycle schedule (the autotuner's pick where it chooses)
    o.set_solver(jv_mode=JV_ANALYTIC, nu1=sv["nu1"], nu2=sv["nu2"], nmg=4,
                 coarse_sweeps=sv["coarse_sweeps"])
    leaf = int(o.leaf_mask().sum())
    o.pc_setup(u0, 1.0, DT)
    rng = np.random.default_rng(0)
    w = rng.standard_normal(u0.size)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        y = o.pc_apply(w)
        w = o.jv_analytic(u0, y, 1.0, DT)
        w /= np.sqrt(max(o.dot(w, w), 1e-300))
        t1 = time.perf_counter()
        if s >= args.warmup:
            times.append(t1 - t0)
    tot = sum(times)
    val = leaf * args.steps / tot / 1e6
    sample = ("one FP64 oracle Krylov iteration (FAC/GMG P^-1 + analytic Jv) per step on %s "
              "(%d leaf cells), %d host threads"
              % ("the full workload" if wl["cpu_n"] is None
                 else "the %d^3 version of the layout" % wl["cpu_n"], leaf, cores))
    line = {
        "impl": "reference", "metric": "Mcell/s of Jv+V-cycle", "value": val, "unit": "Mcell/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "sample_leaf_cells": leaf,
                   "step": "one Krylov iteration"},
        "cpu_baseline": {"value": val, "unit": "Mcell/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": model},
        "e2e": {"value": val, "unit": "Mcell/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def vcycle_bytes_per_cell(h, sweeps):
    """Algorithmic DRAM bytes of one FP32 V-cycle apply per leaf cell, both
    fields: per red-black sweep of a level (the two colours fused, perfect
    neighbour reuse) the 3 face-coefficient arrays, e read and written and
    the rhs, 4 B each: 24 B per cell and field; per level visit the residual
    (e, rhs, 3 coefficients, r written: 24 B), restriction (r read, coarse rhs
    written: 4.5 B) and prolongation (coarse e, e read and written: 8.5 B);
    the coarser levels add 1/8 each; the FP64 input (16 B), the P2 data
    (12 B: three FP32 values) and the FP64 output (16 B) once."""
    nu = int(sweeps[0]) + int(sweeps[1])
    per_field = 24.0 * nu + 24.0 + 4.5 + 8.5
    return 2 * per_field * 8.0 / 7.0 + 16 + 12 + 16


def main():
    global DT
    args = parse()
    DT = WORKLOADS[args.workload]["dt"]
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile:
        return profile_run(args)
    if args.profile_pc:
        return profile_pc_run(args)
    if args.adjoint:
        return adjoint_run(args)
    if args.profile_stencils:
        return profile_stencils_run(args)
    if args.levels_table > 0:
        return levels_table(args)
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    key = args.workload
    wl = WORKLOADS[key]
    h, z, u0 = workload(key)
    rates = nrd.measure_peaks()
    ops = nrd.measure_fp64_ops()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ctx = make_ctx(nrd, h, z, torch, production=True, wl=wl)
    leaf = ctx.nleaf
    # autotuners: stencil tile shape for this hierarchy, and the smoother
    # schedule where the workload does not state one (untimed set-up)
    u_t = torch.from_numpy(u0).cuda()
    tile, _ = ctx.autotune(u_t, u_t, 1.0, DT)
    if wl["solver"] is None:
        sweeps, _ = ctx.autotune_sweeps(u_t, None, DT)
    else:
        sv = wl["solver"]
        sweeps = (sv["nu1"], sv["nu2"], sv["coarse_sweeps"], nrd.SMOOTH_RBGS)
    del u_t

    # production form, timed (replicas: every rank runs the same workload):
    # each implicit step is one launch of the Newton graph
    barrier()
    clk = ClockSampler(local)
    clk.start()
    r = run_steps(ctx, torch, u0, args.steps, args.warmup, flush, timing=False)
    barrier()
    clocks = clk.stop()
    # instrumented repeat of the same steps: CUDA events around every launch
    # group (this runs the host-driven loop, since event records cannot sit
    # inside the graph's loops); source of the per-kernel times below
    rk = run_steps(ctx, torch, u0, args.steps, args.warmup, flush, timing=True)
    value, tot_ms = replicas_value(dist, world, leaf * r["krylov"], sum(r["ms"]), "cuda")

    # rooflines, measured live with CUDA events around each launch group in
    # the instrumented repeat of the timed steps
    kt = rk["kernel"]
    hbm_peak, peak_src = peaks()
    # FP64 pipe issue rate: the measured FP64 FMA rate in instructions
    # (one FMA = one instruction = 2 flops)
    fp64_peak = rates["fp64_tflops"] * 1e3 / 2.0
    fp64_src = ("FP64 FMA rate measured in this run by nrd_measure_peaks, in instructions "
                "(2 per clock per SM x 152 SMs x clock; MEASURED_PEAKS.json has no FP64 figure)")
    traffic = TRAFFIC.get(key, {})
    lin_ms, lin_n = kt["linearise"]
    t_lin = lin_ms / max(lin_n, 1) * 1e-3
    # FP64 work from the formulas' operation counts: each add, subtract,
    # multiply, division and square root one flop (classical counting),
    # against the measured FMA rate in flops (2 per FMA).  Beside it: the
    # divisions and square roots charged at the FMA-equivalents of CUDA's
    # correctly rounded operations (measured; the kernels use refined
    # reciprocals instead, so that figure can exceed 1), and the FP64-pipe
    # instructions the kernels issue against the pipe's issue rate.
    c_div = 2.0 * ops["fma_per_s"] / ops["div_per_s"]
    c_sqrt = 2.0 * ops["fma_per_s"] / ops["sqrt_per_s"]
    flop_peak = 2.0 * ops["fma_per_s"] / 1e9

    def flops(o):
        return o[0] + o[1] + o[2]

    def charged(o):
        return o[0] + c_div * o[1] + c_sqrt * o[2]

    ach = flops(LIN_OPS) * leaf / t_lin / 1e9
    ach_c = charged(LIN_OPS) * leaf / t_lin / 1e9
    ach_inst = LIN_INST_NCU * leaf / t_lin / 1e9
    roof = {"kernel": "k_stencil<ST_LINF> + k_stencil<ST_LINC> (residual + linearisation, "
                      "FP64: every face once, then the cells)", "bound": "alu",
            "achieved": ach, "peak": flop_peak, "unit": "GFLOP/s (FP64)",
            "frac": ach / flop_peak, "traffic": traffic.get("linearise"),
            "per_launch_us": t_lin * 1e6, "launches": lin_n,
            "timing": "CUDA events around each linearisation (its face and cell launches) in "
                      "an instrumented repeat of the timed steps",
            "peak_source": "FP64 FMA rate measured in this run (nrd_measure_fp64_ops), 2 flops "
                           "per FMA; MEASURED_PEAKS.json has no FP64 figure",
            "algorithmic": "%d FP64 flops per leaf cell (%d add/multiply, %d divisions, %d "
                           "square roots, from the formulas) x %d leaf cells"
                           % (flops(LIN_OPS), LIN_OPS[0], LIN_OPS[1], LIN_OPS[2], leaf),
            "division_charged": {"achieved": ach_c, "frac": ach_c / flop_peak,
                                 "per_cell": charged(LIN_OPS),
                                 "flops_per_division": c_div, "flops_per_sqrt": c_sqrt},
            "fp64_instructions": {"per_cell": LIN_INST_NCU, "achieved": ach_inst,
                                  "peak": fp64_peak, "unit": "Ginst/s (FP64 pipe)",
                                  "frac": ach_inst / fp64_peak,
                                  "source": "ncu sm__inst_executed_pipe_fp64 per cell" + (
                                      "" if key == "single256" else
                                      ", captured on the single-level layout at 128^3 and "
                                      "applied to this workload (not captured here: patch "
                                      "boundaries add faces)")},
            "measured_fp64_ops": ops}
    if traffic.get("linearise"):
        tpc = traffic["linearise"] / leaf
        roof["bytes"] = {"dram_per_cell": tpc, "algorithmic_per_cell": LIN_BYTES_PER_CELL,
                         "ratio": tpc / LIN_BYTES_PER_CELL,
                         "residual_only_per_cell": RES_BYTES_PER_CELL,
                         "ratio_to_residual_only": tpc / RES_BYTES_PER_CELL,
                         "why": "the linearisation also writes the frozen Jacobian partials, "
                                "P1 coefficients, coupling partials and P2 data that the "
                                "Krylov iterations and the V-cycle read (FP64 issue, not "
                                "HBM, bounds these kernels)"}
    jv_ms, jv_n = kt["jv"]
    t_jv = jv_ms / max(jv_n, 1) * 1e-3
    ach_jv = flops(JV_OPS) * leaf / t_jv / 1e9
    ach_jv_inst = JV_INST_NCU * leaf / t_jv / 1e9
    gbs_jv = JV_BYTES_PER_CELL * leaf / t_jv / 1e9
    roof_jv = {"kernel": "k_stencil<ST_JVF> (frozen-Jacobian Jv)", "bound": "alu",
               "achieved": ach_jv, "peak": flop_peak, "unit": "GFLOP/s (FP64)",
               "frac": ach_jv / flop_peak, "traffic": traffic.get("jv"),
               "per_launch_us": t_jv * 1e6, "launches": jv_n,
               "algorithmic": "%d FP64 ops per leaf cell x %d leaf cells" % (JV_OPS[0], leaf),
               "fp64_instructions": {"per_cell": JV_INST_NCU, "achieved": ach_jv_inst,
                                     "peak": fp64_peak, "unit": "Ginst/s (FP64 pipe)",
                                     "frac": ach_jv_inst / fp64_peak},
               "hbm": {"achieved": gbs_jv, "peak": hbm_peak, "unit": "GB/s",
                       "frac": gbs_jv / hbm_peak, "peak_source": peak_src,
                       "algorithmic": "%d B per leaf cell" % JV_BYTES_PER_CELL}}
    if traffic.get("jv"):
        tpc = traffic["jv"] / leaf
        roof_jv["bytes"] = {"dram_per_cell": tpc, "algorithmic_per_cell": JV_BYTES_PER_CELL,
                            "ratio": tpc / JV_BYTES_PER_CELL,
                            "analytic_jv_per_cell": RES_BYTES_PER_CELL,
                            "ratio_to_analytic": tpc / RES_BYTES_PER_CELL,
                            "why": "reads the 5 stored FP64 partials per face instead of "
                                   "re-deriving them from E, T and z (40 FP64 instructions "
                                   "per cell instead of about 130)"}
    pc_ms, pc_n = kt["pc_apply"]
    t_pc = pc_ms / max(pc_n, 1) * 1e-3
    vb = vcycle_bytes_per_cell(h, sweeps)
    gbs_pc = vb * leaf / t_pc / 1e9
    roof_pc = {"kernel": "V-cycle apply (FP32 FAC/GMG, every kernel of one P^-1 apply)",
               "bound": "hbm", "achieved": gbs_pc, "peak": hbm_peak, "unit": "GB/s",
               "frac": gbs_pc / hbm_peak, "per_launch_us": t_pc * 1e6, "launches": pc_n,
               "peak_source": peak_src,
               "algorithmic": "%.0f B per leaf cell (fused red-black sweeps, both fields, "
                              "all levels) x %d leaf cells" % (vb, leaf)}

    # plain form beside it
    plain = None
    if not args.no_plain:
        ctxp = make_ctx(nrd, h, z, torch, production=False, wl=wl)
        ctxp.set_params(tile_x=tile[0], tile_y=tile[1], tile_z=tile[2], nu1=sweeps[0],
                        nu2=sweeps[1], coarse_sweeps=sweeps[2], smoother=sweeps[3])
        rp = run_steps(ctxp, torch, u0, args.steps, args.warmup, flush, timing=False)
        pms = sum(rp["ms"])
        plain = {"form": "FD Jv + FP64 V-cycle, Newton loop driven from the host (no "
                         "graphs); the same batched tile kernels (one launch per sweep over "
                         "all patches), not per-patch launches",
                 "ms_per_step": pms / args.steps,
                 "value": leaf * rp["krylov"] / (pms * 1e-3) / 1e6,
                 "krylov_per_step": rp["krylov"] / args.steps,
                 "newton_per_step": rp["newton"] / args.steps}
        del ctxp

    barrier()
    # the same warm-up and timed steps as the device-resident line, so that
    # the two time the same Newton and Krylov mix
    e_ms, e_kry, h2d, d2h = run_e2e(nrd, ctx, torch, u0, args.steps, args.warmup)
    e_val, _ = replicas_value(dist, world, leaf * e_kry, e_ms, "cuda")
    e2e = {"value": e_val, "unit": "Mcell/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    regrid = None
    if not args.no_regrid and wl["regrid"]:
        regrid = regrid_leg(nrd, ctx, torch, h, z, r)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(key, sweeps)

    # kernels executed in the timed region: the Newton graph's kernel nodes
    # times the iterations of their loops (counted by the library), plus the
    # refinement indicators (average-down per covered level, ghost fill, two
    # reduction kernels, the tag kernel), the predictor and the time
    # derivative (one kernel each) per step
    launches = r["kernels"] + args.steps * ((h.nlevels - 1) + 4 + 2)
    line = {
        "metric": "Mcell/s of Jv+V-cycle", "value": value, "unit": "Mcell/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "step_ms": {"min": min(r["ms"]), "median": float(np.median(r["ms"])),
                    "max": max(r["ms"])},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "sizes": wl["sizes"], "base": h.n0[0],
                   "levels": h.nlevels, "leaf_cells": leaf,
                   "patches": sum(h.nboxes), "dt": DT, "newton_rtol": 1e-8,
                   "form": "analytic Jv + FP32 FAC/GMG V-cycle + FGMRES(30)",
                   "tile": list(tile), "sweeps_nu1_nu2_coarse": list(sweeps[:3]),
                   "sweeps_from": "autotuner" if wl["solver"] is None else "workload",
                   "gmg_levels": 4,
                   "smoother": "jacobi" if sweeps[3] == nrd.SMOOTH_JACOBI else "rbgs",
                   "krylov_per_step": r["krylov"] / args.steps,
                   "newton_per_step": r["newton"] / args.steps,
                   "l2": "256 MB buffer written between timed steps" + (
                       "; every state vector (%d MB) is larger than L2" % (16 * ctx.N >> 20)
                       if 16 * ctx.N > 129e6 else ""),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "roofline_jv": roof_jv,
        "roofline_vcycle": roof_pc,
        "measured_rates": rates,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        "plain": plain,
        "speedup_vs_plain": (plain["ms_per_step"] / (tot_ms / args.steps)) if plain else None,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "regrid": regrid,
        "clocks": clocks,
        "gpu_launches": launches,
        "gpu_launches_note": "kernel nodes executed by the Newton graphs plus the predictor, "
                             "time-derivative and tagging kernels, timed steps only",
        "kernel_ms_note": "kernel_ms_per_step from the instrumented repeat (host-driven loop)",
        "instrumented_ms_per_step": sum(rk["ms"]) / args.steps,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
