"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances, each from the arithmetic:
  ghosts                 1e-14 relative (same formulas, different summation order)
  residual, analytic Jv  |gpu - oracle| <= 1e-12 * S_cell, S_cell the sum of
                         absolute values of the cell's terms (oracle-computed):
                         FP64 rounding of a sum of O(10) terms is ~1e-15 S_cell,
                         so the bound leaves a factor ~1000 for reordering
  FD Jv                  8 eps_mach S_cell / |eps| (rounding of F(u + eps v)
                         amplified by 1/eps) + 1e-12 S_jv
  FP64 V-cycle           1e-11 of max |y| (same algorithm, different rounding,
                         amplified by the V-cycle's few sweeps)
  FP32 V-cycle           2e-4 of max |y| (FP32 rounding, 6e-8, amplified by
                         the operator's condition on the coarse grids)
  converged step         1e-8 relative per cell and field (Newton rtol 1e-10 on
                         both sides: two correct solves then agree to ~1e-11)
  tags                   equal, except where an indicator lies within 1e-12
                         of its threshold (the GPU compares without dividing)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle, JV_ANALYTIC as O_AN, JV_FD as O_FD, LIM_PAPER_LITERAL  # noqa: E402
from paper_1302_6303_gb300 import workloads as W  # noqa: E402
from stepcheck import per_cell_rel  # noqa: E402

EPS = 2.0 ** -52


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


def auto_nmg(h, cap=4):
    m = 1
    while m < cap and all(n % (1 << m) == 0 for n in h.n0):
        m += 1
    return m


def make(nrd, h, z, limiter=0, **kw):
    kw.setdefault("nmg", auto_nmg(h))
    ctx = nrd.Context(limiter=limiter, **kw)
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z.astype(np.float32)))
    o = Oracle(h, z, limiter=limiter)
    return ctx, o


CASES = {
    "single32": lambda: W.config_single_level(32, seed=1, cube_side=8),
    "ragged": lambda: (W.uniform((20, 12, 7)),
                       W.material_from_cubes(W.uniform((20, 12, 7)), [((3, 2, 1), 4, 10.0)])),
    "one_cell": lambda: (W.uniform(1), np.array([3.0], np.float32)),
    "tiny2": lambda: (W.tiny_amr(8), W.material_from_cubes(W.tiny_amr(8), [((2, 2, 2), 3, 10.0)])),
    "tiny3": lambda: (W.tiny_amr(8, True),
                      W.material_from_cubes(W.tiny_amr(8, True), [((3, 3, 3), 3, 10.0)])),
    "boundary": lambda: (W.boundary_amr(8),
                         W.material_from_cubes(W.boundary_amr(8), [((0, 1, 1), 2, 10.0)])),
    "amr2_16": lambda: W.config_amr2(16, seed=3, band=4, ncubes=4),
}


def _state(h, seed=2):
    return W.front_state(h, seed=seed, noise=0.1)


@pytest.mark.parametrize("name", list(CASES))
def test_ghosts(nrd, name):
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z)
    u = _state(h)
    gE, gT, gz = ctx.ghost_fill(dev(u))
    oE, oT, oz = o.ghosts(u)
    np.testing.assert_allclose(gE.cpu().numpy(), oE, rtol=1e-14, atol=0)
    np.testing.assert_allclose(gT.cpu().numpy(), oT, rtol=1e-14, atol=0)
    np.testing.assert_array_equal(gz.cpu().numpy(), oz)


@pytest.mark.parametrize("limiter", [0, LIM_PAPER_LITERAL])
@pytest.mark.parametrize("name", list(CASES))
def test_residual(nrd, name, limiter):
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z, limiter=limiter)
    u = _state(h)
    rng = np.random.default_rng(4)
    b = u * (1 + 0.05 * rng.uniform(-1, 1, u.size))
    a0, dt = 1.5, 3e-3
    F = ctx.residual(dev(u), dev(b), a0, dt).cpu().numpy()
    Fo = o.residual(u, b, a0, dt)
    S = o.residual_scale(u, b, a0, dt)
    err = np.abs(F - Fo)
    assert np.all(err <= 1e-12 * S + 1e-300), (err / np.maximum(S, 1e-300)).max()
    leaf = np.concatenate([o.leaf_mask()] * 2)
    assert np.all(F[~leaf] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_jv_analytic(nrd, name):
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z)
    u = _state(h)
    v = W.random_direction(h, 7)
    a0, dt = 1.0, 2e-3
    J = ctx.jv(dev(u), dev(v), a0, dt, mode=nrd.JV_ANALYTIC).cpu().numpy()
    Jo = o.jv_analytic(u, v, a0, dt)
    S = o.jv_scale(u, v, a0, dt)
    err = np.abs(J - Jo)
    assert np.all(err <= 1e-12 * S + 1e-300), (err / np.maximum(S, 1e-300)).max()


@pytest.mark.parametrize("name", list(CASES))
def test_jv_fd_and_eps(nrd, name):
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z)
    u = _state(h)
    v = W.random_direction(h, 8)
    a0, dt = 1.0, 2e-3
    b = u.copy()
    F0 = o.residual(u, b, a0, dt)
    eps_g = ctx.fd_eps(dev(u), dev(v))
    eps_o = o.fd_eps(u, v)
    assert abs(eps_g - eps_o) <= 1e-13 * abs(eps_o)
    J = ctx.jv(dev(u), dev(v), a0, dt, mode=nrd.JV_FD, b=dev(b), F0=dev(F0)).cpu().numpy()
    Jo, eps = o.jv_fd(u, v, b, a0, dt, F0=F0)
    up = u + eps * v
    S = o.residual_scale(up, b, a0, dt)
    Sj = o.jv_scale(u, v, a0, dt)
    tol = 8 * EPS * S / abs(eps) + 1e-12 * Sj
    assert np.all(np.abs(J - Jo) <= tol), (np.abs(J - Jo) / tol).max()


@pytest.mark.parametrize("name", ["single32", "tiny3", "amr2_16"])
def test_dot(nrd, name):
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z)
    x = W.random_direction(h, 1)
    y = W.random_direction(h, 2)
    d = ctx.dot(dev(x), dev(y))
    do = o.dot(x, y)
    scale = o.dot(np.abs(x), np.abs(y))
    assert abs(d - do) <= 1e-14 * scale


@pytest.mark.parametrize("name", ["single32", "tiny3", "boundary", "amr2_16"])
def test_tag(nrd, name):
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z)
    u = _state(h)
    for thr in [(0.5, np.inf, np.inf), (np.inf, 0.3, np.inf), (np.inf, np.inf, 0.1)]:
        t = ctx.tag(dev(u), *thr).cpu().numpy()
        to = o.tag(u, *thr)
        # the GPU decides without divisions (cross-multiplied comparisons),
        # the oracle compares the divided indicator: a tag may differ only
        # where the indicator is within rounding of its threshold
        ind = o.tag_values(u)
        for bit in range(3):
            diff = ((t >> bit) & 1) != ((to >> bit) & 1)
            if diff.any():
                near = np.abs(ind[diff, bit] - thr[bit]) <= 1e-12 * thr[bit]
                assert near.all(), (bit, ind[diff, bit][~near][:5], thr[bit])


# red-black schedules (nu1, nu2, coarse sweeps): V(2,2); V(1,0), where the
# up-leg of the FAC cycle only prolongs (no post-smoothing, no residuals);
# V(1,1); V(3,3), the 256^3 workload's
RB_SCHED = [(2, 2, 4), (1, 0, 2), (1, 1, 2), (3, 3, 6)]


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4)])
@pytest.mark.parametrize("sched", RB_SCHED)
@pytest.mark.parametrize("name", ["single32", "tiny2", "tiny3", "boundary", "amr2_16"])
def test_precond_apply(nrd, name, sched, prec, tol):
    h, z = CASES[name]()
    nmg = 3 if h.n0[0] >= 16 else 2
    nu1, nu2, csw = sched
    ctx, o = make(nrd, h, z, pc_precision=prec, nmg=nmg, nu1=nu1, nu2=nu2, coarse_sweeps=csw)
    o.set_solver(nmg=nmg, nu1=nu1, nu2=nu2, coarse_sweeps=csw)
    u = _state(h)
    a0, dt = 1.2, 5e-3
    ctx.precond_setup(dev(u), a0, dt)
    o.pc_setup(u, a0, dt)
    w = W.random_direction(h, 5)
    y = ctx.precond_apply(dev(w)).cpu().numpy()
    yo = o.pc_apply(w)
    assert np.abs(y - yo).max() <= tol * np.abs(yo).max(), np.abs(y - yo).max() / np.abs(yo).max()


@pytest.mark.parametrize("jv", ["fd", "analytic"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["single32", "tiny2", "amr2_16"])
def test_newton_step(nrd, name, prec, jv):
    h, z = CASES[name]()
    nmg = 3 if h.n0[0] >= 16 else 2
    mode = nrd.JV_FD if jv == "fd" else nrd.JV_ANALYTIC
    ctx, o = make(nrd, h, z, pc_precision=prec, nmg=nmg, jv_mode=mode, rtol=1e-10, restart=30)
    o.set_solver(nmg=nmg, jv_mode=O_FD if jv == "fd" else O_AN, rtol=1e-10)
    u0 = W.initial_state(h)
    # a warmed-up state: the Marshak front has entered
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    un = dev(u0)
    u = un.clone()
    st = ctx.step(u, un, None, 1e-3)
    uo, sto = o.newton(u0.copy(), u0.copy(), 1.0, 1e-3)
    assert st["status"] == 0 and sto["status"] == 0
    rel = per_cell_rel(u.cpu().numpy(), uo, o.leaf_mask())
    assert rel <= 1e-8, (rel, st, sto)


def test_bdf2_step_matches_oracle(nrd):
    h, z = CASES["tiny2"]()
    ctx, o = make(nrd, h, z, pc_precision=0, nmg=2, jv_mode=nrd.JV_ANALYTIC, rtol=1e-10)
    o.set_solver(nmg=2, jv_mode=O_AN, rtol=1e-10)
    u1 = W.front_state(h, seed=1, noise=0.0, front=0.1)
    u0 = W.front_state(h, seed=1, noise=0.0, front=0.08)
    dt, dtp = 1e-3, 5e-4
    al = dt / dtp
    a0 = (1 + 2 * al) / (1 + al)
    b = (1 + al) * u1 - al * al / (1 + al) * u0
    u = dev(u1)
    st = ctx.step(u, dev(u1), dev(u0), dt, dtp)
    uo, sto = o.newton(u1.copy(), b, a0, dt)
    rel = per_cell_rel(u.cpu().numpy(), uo, o.leaf_mask())
    assert st["status"] == 0 and rel <= 1e-8, rel


def test_full_size_residual_and_jv(nrd):
    """The 2-level benchmark workload (64^3 base + fine patches over the
    Marshak band, 491,520 leaf cells) in the benchmark's launch configuration
    (8x8x4 stencil tiles; the linearisation's face and cell launches and the
    frozen Jv the Krylov loop uses), and the residual-only and tangent
    forms: every cell checked."""
    h, z = W.config_amr2(64, seed=0)
    ctx, o = make(nrd, h, z, tile_x=8, tile_y=8, tile_z=4)
    u = W.front_state(h, seed=3, noise=0.05)
    v = W.random_direction(h, 4)
    a0, dt = 1.0, 5e-4
    Fo = o.residual(u, u.copy(), a0, dt)
    S = o.residual_scale(u, u.copy(), a0, dt)
    Jo = o.jv_analytic(u, v, a0, dt)
    Sj = o.jv_scale(u, v, a0, dt)
    F = ctx.residual(dev(u), dev(u), a0, dt).cpu().numpy()
    assert np.all(np.abs(F - Fo) <= 1e-12 * S + 1e-300)
    J = ctx.jv(dev(u), dev(v), a0, dt, mode=nrd.JV_ANALYTIC).cpu().numpy()
    assert np.all(np.abs(J - Jo) <= 1e-12 * Sj + 1e-300)
    F = ctx.linearise(dev(u), dev(u), a0, dt).cpu().numpy()
    assert np.all(np.abs(F - Fo) <= 1e-12 * S + 1e-300)
    J = ctx.jv(dev(u), dev(v), a0, dt, mode=nrd.JV_FROZEN).cpu().numpy()
    assert np.all(np.abs(J - Jo) <= 1e-12 * Sj + 1e-300)


def test_errors_are_reported(nrd):
    ctx = nrd.Context()
    with pytest.raises(nrd.NrdError) as e:
        ctx.residual(dev(np.ones(2)), dev(np.ones(2)), 1.0, 1.0)
    assert e.value.code == nrd.ESTATE
    # misaligned fine box
    with pytest.raises(nrd.NrdError) as e:
        ctx.set_hierarchy([1, 1], [0, 0, 0, 7, 7, 7, 1, 2, 2, 4, 5, 5], [1, 0, 0, 0, 0, 0],
                          [1.0, 0, 0, 0, 0, 0])
    assert e.value.code == nrd.EINVAL
    # improperly nested third level
    h = W.tiny_amr(8)
    boxes = h.boxes_flat() + [0, 0, 0, 3, 3, 3]
    with pytest.raises(nrd.NrdError) as e:
        ctx.set_hierarchy(h.nboxes + [1], boxes, h.bc_type, h.bc_R)
    assert e.value.code == nrd.EINVAL


@pytest.mark.parametrize("name", list(CASES))
def test_linearise_and_frozen_jv(nrd, name):
    """nrd_linearise returns the residual and freezes the exact Jacobian: the
    frozen Jv equals the oracle's tangent (dual numbers) within 1e-12 S."""
    h, z = CASES[name]()
    ctx, o = make(nrd, h, z, pc_precision=0)
    u = _state(h)
    v = W.random_direction(h, 11)
    b = u * 0.97
    a0, dt = 1.3, 2e-3
    F = ctx.linearise(dev(u), dev(b), a0, dt).cpu().numpy()
    Fo = o.residual(u, b, a0, dt)
    S = o.residual_scale(u, b, a0, dt)
    assert np.all(np.abs(F - Fo) <= 1e-12 * S + 1e-300)
    J = ctx.jv(dev(u), dev(v), a0, dt, mode=nrd.JV_FROZEN).cpu().numpy()
    Jo = o.jv_analytic(u, v, a0, dt)
    Sj = o.jv_scale(u, v, a0, dt)
    err = np.abs(J - Jo)
    assert np.all(err <= 1e-12 * Sj + 1e-300), (err / np.maximum(Sj, 1e-300)).max()
    leaf = np.concatenate([o.leaf_mask()] * 2)
    assert np.all(J[~leaf] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_residual_bitwise_equals_linearise(nrd, name):
    """The residual-only evaluation and the linearisation share their face
    and cell arithmetic: the same F bit for bit (the Newton loop evaluates F
    alone at a predicted last iterate and relies on this)."""
    h, z = CASES[name]()
    ctx, _ = make(nrd, h, z, pc_precision=0)
    u = _state(h)
    b = u * 0.97
    a0, dt = 1.3, 2e-3
    F1 = ctx.residual(dev(u), dev(b), a0, dt)
    F2 = ctx.linearise(dev(u), dev(b), a0, dt)
    assert torch.equal(F1, F2)


@pytest.mark.parametrize("name", ["single32", "tiny3", "boundary", "amr2_16"])
def test_linearise_sets_up_preconditioner(nrd, name):
    h, z = CASES[name]()
    nmg = auto_nmg(h, 3)
    ctx, o = make(nrd, h, z, pc_precision=0, nmg=nmg)
    o.set_solver(nmg=nmg, nu1=2, nu2=2, coarse_sweeps=4)
    u = _state(h)
    a0, dt = 1.2, 5e-3
    ctx.linearise(dev(u), dev(u), a0, dt)
    o.pc_setup(u, a0, dt)
    w = W.random_direction(h, 6)
    y = ctx.precond_apply(dev(w)).cpu().numpy()
    yo = o.pc_apply(w)
    assert np.abs(y - yo).max() <= 1e-11 * np.abs(yo).max()


def test_frozen_jv_requires_linearise(nrd):
    h, z = CASES["single32"]()
    ctx, _ = make(nrd, h, z)
    u = dev(_state(h))
    with pytest.raises(nrd.NrdError) as e:
        ctx.jv(u, u, 1.0, 1e-3, mode=nrd.JV_FROZEN)
    assert e.value.code == nrd.ESTATE


SHAPES = [(32, 4, 4), (32, 8, 4), (32, 4, 8), (32, 2, 4), (16, 8, 4), (16, 4, 8), (16, 8, 8),
          (16, 4, 4), (8, 8, 8), (8, 8, 4)]


@pytest.mark.parametrize("shape", SHAPES)
def test_every_tile_shape(nrd, shape):
    """Residual, frozen Jv and one FP64 V-cycle agree with the oracle for every
    compiled tile shape (ragged tiles on 16-wide fine patches included)."""
    h, z = CASES["amr2_16"]()
    tx, ty, tz = shape
    ctx, o = make(nrd, h, z, pc_precision=0, nmg=3, tile_x=tx, tile_y=ty, tile_z=tz)
    o.set_solver(nmg=3)
    u = _state(h)
    a0, dt = 1.0, 2e-3
    F = ctx.linearise(dev(u), dev(u), a0, dt).cpu().numpy()
    S = o.residual_scale(u, u.copy(), a0, dt)
    assert np.all(np.abs(F - o.residual(u, u.copy(), a0, dt)) <= 1e-12 * S + 1e-300)
    v = W.random_direction(h, 3)
    J = ctx.jv(dev(u), dev(v), a0, dt, mode=nrd.JV_FROZEN).cpu().numpy()
    Sj = o.jv_scale(u, v, a0, dt)
    assert np.all(np.abs(J - o.jv_analytic(u, v, a0, dt)) <= 1e-12 * Sj + 1e-300)
    o.pc_setup(u, a0, dt)
    y = ctx.precond_apply(dev(v)).cpu().numpy()
    yo = o.pc_apply(v)
    assert np.abs(y - yo).max() <= 1e-11 * np.abs(yo).max()


def test_autotune_keeps_parity(nrd):
    h, z = CASES["amr2_16"]()
    ctx, o = make(nrd, h, z, pc_precision=0, nmg=3)
    u = _state(h)
    shape, ms = ctx.autotune(dev(u), dev(u), 1.0, 2e-3)
    assert tuple(shape) in SHAPES and ms > 0
    F = ctx.residual(dev(u), dev(u), 1.0, 2e-3).cpu().numpy()
    S = o.residual_scale(u, u.copy(), 1.0, 2e-3)
    assert np.all(np.abs(F - o.residual(u, u.copy(), 1.0, 2e-3)) <= 1e-12 * S + 1e-300)


def test_sweep_autotuner_keeps_solution(nrd):
    h, z = CASES["amr2_16"]()
    ctx, o = make(nrd, h, z, pc_precision=1, nmg=3, jv_mode=nrd.JV_ANALYTIC, rtol=1e-10)
    o.set_solver(nmg=3, jv_mode=O_AN, rtol=1e-10)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    nu, ms = ctx.autotune_sweeps(dev(u0), None, 1e-3)
    assert nu[:3] in [(1, 0, 2), (1, 1, 2), (2, 1, 3), (2, 2, 4), (3, 3, 6)] and ms > 0
    assert nu[3] in (nrd.SMOOTH_RBGS, nrd.SMOOTH_JACOBI)
    assert ctx.params.smoother == nu[3]
    u = dev(u0)
    st = ctx.step(u, dev(u0), None, 1e-3)
    uo, sto = o.newton(u0.copy(), u0.copy(), 1.0, 1e-3)
    rel = per_cell_rel(u.cpu().numpy(), uo, o.leaf_mask())
    assert st["status"] == 0 and rel <= 1e-8, rel


# ------------------------------------------------- graph-captured Newton solve
def _graph_pair(nrd, h, z, **kw):
    kw.setdefault("nmg", auto_nmg(h))
    out = []
    for g in (1, 0):
        ctx = nrd.Context(graph=g, **kw)
        ctx.set_hierarchy_from(h)
        ctx.set_material(dev(z.astype(np.float32)))
        out.append(ctx)
    return out


@pytest.mark.parametrize("name", ["tiny2", "tiny3", "amr2_16", "ragged"])
def test_graph_newton_matches_host_loop(nrd, name):
    """The whole Newton solve as one CUDA graph (device-side loops) gives the
    host-driven loop's iterates: the same Newton / Krylov counts and the same
    converged state (BE step, then a BDF2 step with another dt on the same
    instantiated graph)."""
    h, z = CASES[name]()
    cg, ch = _graph_pair(nrd, h, z, rtol=1e-10, jv_mode=nrd.JV_ANALYTIC)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    leaf = ~h.covered_mask()
    res = []
    for ctx in (cg, ch):
        un = dev(u0)
        u1 = un.clone()
        s1 = ctx.step(u1, un, None, 1e-3)
        u2 = u1.clone()
        s2 = ctx.step(u2, u1, un, 7e-4, 1e-3)
        res.append((u1.cpu().numpy(), u2.cpu().numpy(), s1, s2))
    (g1, g2, gs1, gs2), (h1, h2, hs1, hs2) = res
    for a, b in ((g1, h1), (g2, h2)):
        rel = per_cell_rel(a, b, leaf)
        assert rel <= 1e-8, rel
    for sg, sh in ((gs1, hs1), (gs2, hs2)):
        assert sg["status"] == 0 and sh["status"] == 0
        assert abs(sg["newton_its"] - sh["newton_its"]) <= 1
        assert abs(sg["krylov_its"] - sh["krylov_its"]) <= 2
        assert abs(sg["fnorm0"] - sh["fnorm0"]) <= 1e-12 * sh["fnorm0"]


def test_graph_newton_restarts_and_caps(nrd):
    """GMRES restarts (restart length 2) and the Newton cap inside the graph:
    the restarted solve converges to the host loop's state, and a capped solve
    reports NRD_ENONCONV in both forms."""
    h, z = CASES["amr2_16"]()
    cg, ch = _graph_pair(nrd, h, z, rtol=1e-10, restart=2, pc_precision=nrd.PC_F32)
    u0 = W.front_state(h, seed=2, noise=0.02, front=0.2, width=0.05)
    outs = []
    for ctx in (cg, ch):
        u = dev(u0)
        st = ctx.step(u, dev(u0), None, 2e-3)
        outs.append((u.cpu().numpy(), st))
    (ug, sg), (uh, sh) = outs
    assert sg["status"] == 0 and sh["status"] == 0
    assert sg["krylov_its"] > 2 * sg["newton_its"] - 1 or sh["krylov_its"] > 2 * sh["newton_its"] - 1
    assert per_cell_rel(ug, uh, ~h.covered_mask()) <= 1e-8
    for ctx in (cg, ch):
        ctx.set_params(max_newton=1, rtol=1e-14)
        u = dev(u0)
        st = ctx.step(u, dev(u0), None, 2e-3, check=False)
        assert st["status"] == nrd.ENONCONV and st["newton_its"] == 1


def test_refined_reciprocals_error_bound(nrd):
    """The linearisation's refined reciprocal and reciprocal square root
    (PTX approximate seeds, second-order series correction) against CUDA's
    correctly rounded 1/x, 1/sqrt(x): relative error within a few units in
    the last place over 26 decades, and the rounded operations at the range
    edges."""
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-13, 13, 200000),
                        [1e-305, 1e-300, 1e300, 1e305, 1.0, 0.5, 2.0]])
    out = nrd.check_fastmath(dev(x)).cpu().numpy()
    r_err = np.abs(out[0] - out[1]) / out[1]
    s_err = np.abs(out[2] - out[3]) / out[3]
    assert r_err.max() <= 1e-15 and s_err.max() <= 1e-15, (r_err.max(), s_err.max())
    assert out[0][-4] == out[1][-4] and out[2][-4] == out[3][-4]   # 1e305: rounded path


def test_integer_narrowing_bit_identical(nrd):
    """The stencil's FP64 -> FP32 narrowing from integer instructions against
    CUDA's conversion, bit for bit: random values over the whole FP64 range,
    random bit patterns (zero, subnormals, inf, NaN included), and doubles whose
    29 dropped bits sit at and around the rounding tie with an even and an odd
    kept lsb, at the float range edges and with a mantissa carry into the
    exponent (up to overflow).  The normal-range results also equal numpy's
    round-to-nearest-even cast."""
    rng = np.random.default_rng(3)
    xs = [rng.standard_normal(200000) * 10.0 ** rng.uniform(-50, 50, 200000)]
    bits = rng.integers(0, 2 ** 63, 200000, dtype=np.uint64)
    bits |= rng.integers(0, 2, 200000, dtype=np.uint64) << np.uint64(63)
    xs.append(bits.view(np.float64))
    tops = np.array([0x3F800000, 0x3F800001, 0x3FFFFFFF, 0x7F7FFFFF, 0x7F7FFFFE, 0x00800000,
                     0x00800001, 0x007FFFFF, 0x00000001], dtype=np.uint32)
    base = tops.view(np.float32).astype(np.float64).view(np.uint64)
    low = np.array([0, 1, 0x0FFFFFFF, 0x10000000, 0x10000001, 0x1FFFFFFF], dtype=np.uint64)
    edge = ((base[:, None] & ~np.uint64(0x1FFFFFFF)) | low[None, :]).ravel()
    edge = np.concatenate([edge, edge | (np.uint64(1) << np.uint64(63))])
    xs.append(edge.view(np.float64))
    xs.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38,
                        3.4028235677973362e38, 1.1754942807573643e-38, 5e-324]))
    x = np.concatenate(xs)
    out = nrd.check_narrow(dev(x)).cpu().numpy()
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))
    with np.errstate(over="ignore", invalid="ignore"):
        ref = x.astype(np.float32)
    normal = np.isfinite(ref) & (np.abs(ref) >= np.finfo(np.float32).tiny)
    assert np.array_equal(out[0][normal].view(np.uint32), ref[normal].view(np.uint32))
