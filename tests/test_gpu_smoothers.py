"""Smoother variants of the V-cycle (Sec. 4.3): the damped point Jacobi
smoother and block (x-line) Gauss-Seidel on the GPU against the FP64 oracle,
and the iteration counts of the smoothers and sweep schedules on one
implicit step.

Tolerances as in test_gpu_parity: FP64 V-cycle 1e-11 of max |y| (same
algorithm, different rounding), FP32 V-cycle 2e-4, converged step 1e-8
relative (Newton rtol 1e-10 on both sides).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle, JV_ANALYTIC as O_AN  # noqa: E402
from paper_1302_6303_gb300 import workloads as W  # noqa: E402
from stepcheck import per_cell_rel  # noqa: E402

OMEGA = 6.0 / 7.0


@pytest.fixture(scope="session")
def nrd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = {
    "single16": lambda: W.config_single_level(16, seed=1, cube_side=4),
    "tiny2": lambda: (W.tiny_amr(8), W.material_from_cubes(W.tiny_amr(8), [((2, 2, 2), 3, 10.0)])),
    "tiny3": lambda: (W.tiny_amr(8, True),
                      W.material_from_cubes(W.tiny_amr(8, True), [((3, 3, 3), 3, 10.0)])),
    "boundary": lambda: (W.boundary_amr(8),
                         W.material_from_cubes(W.boundary_amr(8), [((0, 1, 1), 2, 10.0)])),
    "amr2_16": lambda: W.config_amr2(16, seed=3, band=4, ncubes=4),
}


def make(nrd, h, z, **kw):
    ctx = nrd.Context(**kw)
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z.astype(np.float32)))
    o = Oracle(h, z)
    return ctx, o


# sweep schedules (nu1, nu2, coarse): even and odd post-smoothing counts take
# the two buffer orders of the Jacobi sweeps; nu2 = 0 adds the level-0
# correction without a smoothing pass
SCHED = [(2, 2, 4), (1, 1, 2), (1, 3, 3), (2, 0, 1)]


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4)])
@pytest.mark.parametrize("sched", SCHED)
@pytest.mark.parametrize("name", list(CASES))
def test_jacobi_precond_apply(nrd, name, sched, prec, tol):
    h, z = CASES[name]()
    nmg = 3 if h.n0[0] >= 16 else 2
    nu1, nu2, csw = sched
    ctx, o = make(nrd, h, z, pc_precision=prec, nmg=nmg, nu1=nu1, nu2=nu2, coarse_sweeps=csw,
                  smoother=nrd.SMOOTH_JACOBI, omega=OMEGA)
    o.set_solver(nmg=nmg, nu1=nu1, nu2=nu2, coarse_sweeps=csw)
    o.set_smoother(1, OMEGA)
    u = W.front_state(h, seed=2, noise=0.1)
    a0, dt = 1.2, 5e-3
    ctx.precond_setup(dev(u), a0, dt)
    o.pc_setup(u, a0, dt)
    w = W.random_direction(h, 5)
    y = ctx.precond_apply(dev(w)).cpu().numpy()
    yo = o.pc_apply(w)
    err = np.abs(y - yo).max() / np.abs(yo).max()
    assert err <= tol, err


LINE_CASES = dict(CASES, single32=lambda: W.config_single_level(32, seed=1, cube_side=8),
                  odd=lambda: (W.uniform((12, 10, 6)),
                               W.material_from_cubes(W.uniform((12, 10, 6)),
                                                     [((2, 1, 1), 4, 10.0)])))


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4)])
@pytest.mark.parametrize("sched", [(2, 2, 4), (1, 1, 2), (1, 3, 3)])
@pytest.mark.parametrize("name", list(LINE_CASES))
def test_line_gs_precond_apply(nrd, name, sched, prec, tol):
    """Block Gauss-Seidel with x-line blocks (reading R26) on the GMG box
    levels, point red-black sweeps on the patch levels: the V-cycle against
    the oracle's; single levels (including a 32^3 box whose levels have TMA
    maps, which this smoother does not use, and an odd-sized box) and
    2- and 3-level hierarchies."""
    h, z = LINE_CASES[name]()
    nmg = 3 if min(h.n0) >= 16 else (2 if all(n % 2 == 0 for n in h.n0) else 1)
    nu1, nu2, csw = sched
    ctx, o = make(nrd, h, z, pc_precision=prec, nmg=nmg, nu1=nu1, nu2=nu2, coarse_sweeps=csw,
                  smoother=nrd.SMOOTH_LINE)
    o.set_solver(nmg=nmg, nu1=nu1, nu2=nu2, coarse_sweeps=csw)
    o.set_smoother(2)
    u = W.front_state(h, seed=2, noise=0.1)
    a0, dt = 1.2, 5e-3
    ctx.precond_setup(dev(u), a0, dt)
    o.pc_setup(u, a0, dt)
    w = W.random_direction(h, 5)
    y = ctx.precond_apply(dev(w)).cpu().numpy()
    yo = o.pc_apply(w)
    err = np.abs(y - yo).max() / np.abs(yo).max()
    assert err <= tol, err


@pytest.mark.parametrize("name", ["single16", "amr2_16"])
def test_line_gs_newton_step(nrd, name):
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z, pc_precision=1, nmg=3, jv_mode=nrd.JV_ANALYTIC, rtol=1e-10,
                  smoother=nrd.SMOOTH_LINE)
    o.set_solver(nmg=3, jv_mode=O_AN, rtol=1e-10)
    o.set_smoother(2)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    u = dev(u0)
    st = ctx.step(u, dev(u0), None, 1e-3)
    uo, sto = o.newton(u0.copy(), u0.copy(), 1.0, 1e-3)
    assert st["status"] == 0 and sto["status"] == 0
    rel = per_cell_rel(u.cpu().numpy(), uo, o.leaf_mask())
    assert rel <= 1e-8, rel


def test_jacobi_large_gmg_tail(nrd):
    """A base box deep enough for the one-CTA coarse end of the GMG V-cycle
    (FP32): Jacobi sweeps there from shared memory against the oracle."""
    h, z = W.config_single_level(32, seed=1, cube_side=8)
    ctx, o = make(nrd, h, z, pc_precision=1, nmg=4, nu1=1, nu2=1, coarse_sweeps=3,
                  smoother=nrd.SMOOTH_JACOBI, omega=0.8)
    o.set_solver(nmg=4, nu1=1, nu2=1, coarse_sweeps=3)
    o.set_smoother(1, 0.8)
    u = W.front_state(h, seed=4, noise=0.1)
    ctx.precond_setup(dev(u), 1.0, 2e-3)
    o.pc_setup(u, 1.0, 2e-3)
    w = W.random_direction(h, 9)
    y = ctx.precond_apply(dev(w)).cpu().numpy()
    yo = o.pc_apply(w)
    assert np.abs(y - yo).max() <= 2e-4 * np.abs(yo).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["tiny2", "amr2_16"])
def test_jacobi_newton_step(nrd, name, prec):
    h, z = CASES[name]()
    nmg = 3 if h.n0[0] >= 16 else 2
    ctx, o = make(nrd, h, z, pc_precision=prec, nmg=nmg, jv_mode=nrd.JV_ANALYTIC, rtol=1e-10,
                  smoother=nrd.SMOOTH_JACOBI, omega=OMEGA)
    o.set_solver(nmg=nmg, jv_mode=O_AN, rtol=1e-10)
    o.set_smoother(1, OMEGA)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    u = dev(u0)
    st = ctx.step(u, dev(u0), None, 1e-3)
    uo, sto = o.newton(u0.copy(), u0.copy(), 1.0, 1e-3)
    assert st["status"] == 0 and sto["status"] == 0
    rel = per_cell_rel(u.cpu().numpy(), uo, o.leaf_mask())
    assert rel <= 1e-8, rel


def test_smoother_iteration_counts(nrd, capsys):
    """One BE step of a 2-level Marshak-band state with the smoothers and
    schedules of Sec. 4.3: red-black Gauss-Seidel V(1,1) and V(2,2) with
    4-level GMG on the base, the paper's V(1,0) with smoothing only on the
    coarsest AMR level, damped Jacobi V(1,1) and V(2,2).  Every variant
    converges to the same solution; the counts are printed (a report, not a
    pin: they depend on the state)."""
    h, z = W.config_amr2(32, seed=5, band=4, ncubes=8)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    variants = [
        ("RB-GS V(1,1), 4-level GMG", dict(nu1=1, nu2=1, nmg=4, coarse_sweeps=2)),
        ("RB-GS V(2,2), 4-level GMG", dict(nu1=2, nu2=2, nmg=4, coarse_sweeps=4)),
        ("RB-GS V(1,0), smoothing-only coarsest", dict(nu1=1, nu2=0, nmg=1, coarse_sweeps=1)),
        ("Jacobi V(1,1), 4-level GMG", dict(nu1=1, nu2=1, nmg=4, coarse_sweeps=2,
                                              smoother=nrd.SMOOTH_JACOBI, omega=OMEGA)),
        ("Jacobi V(2,2), 4-level GMG", dict(nu1=2, nu2=2, nmg=4, coarse_sweeps=4,
                                              smoother=nrd.SMOOTH_JACOBI, omega=OMEGA)),
        ("x-line block GS V(1,1), 4-level GMG", dict(nu1=1, nu2=1, nmg=4, coarse_sweeps=2,
                                                     smoother=nrd.SMOOTH_LINE)),
    ]
    sols, rows = [], []
    for label, kw in variants:
        ctx = nrd.Context(jv_mode=nrd.JV_ANALYTIC, pc_precision=nrd.PC_F32, rtol=1e-10,
                          max_krylov=2000, **kw)
        ctx.set_hierarchy_from(h)
        ctx.set_material(dev(z.astype(np.float32)))
        u = dev(u0)
        st = ctx.step(u, dev(u0), None, 5e-4)
        assert st["status"] == 0, (label, st)
        sols.append(u.cpu().numpy())
        rows.append((label, st["newton_its"], st["krylov_its"]))
    leaf = ~h.covered_mask()
    for s in sols[1:]:
        assert per_cell_rel(s, sols[0], leaf) <= 1e-7
    with capsys.disabled():
        print("\nsmoother comparison (one BE step, base 32^3 + Marshak band, rtol 1e-10):")
        for label, nn, nk in rows:
            print("  %-40s Newton %2d  Krylov %3d" % (label, nn, nk))
