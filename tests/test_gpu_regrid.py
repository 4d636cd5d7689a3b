"""Regridding (Sec. 5) on the GPU path against the oracle.

Clustering is integer work: the boxes of nrd_regrid_boxes must equal the
oracle's exactly.  The transfer is two FP64 operations per axis (a minmod of
differences, a multiply-add): 1e-14 of max |u| covers the fused multiply-add
the device may use where the oracle rounds twice.  The warm-restart re-solve
is a converged Newton step: 1e-8 relative, as for the other steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import regrid as R  # noqa: E402
from oracle.oracle import Oracle, JV_ANALYTIC as O_AN  # noqa: E402
from paper_1302_6303_gb300 import workloads as W  # noqa: E402
from regrid_cases import golden_cases, load_case, random_hierarchy  # noqa: E402
from stepcheck import per_cell_rel  # noqa: E402


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


def ctx_for(nrd, h, z=None, **kw):
    kw.setdefault("nmg", auto_nmg(h))
    ctx = nrd.Context(**kw)
    ctx.set_hierarchy_from(h)
    if z is None:
        z = np.ones(h.ncells, np.float32)
    ctx.set_material(dev(np.asarray(z, np.float32)))
    return ctx


def as_lists(levels):
    return [[(tuple(lo), tuple(hi)) for lo, hi in lev] for lev in levels]


@pytest.mark.parametrize("path", golden_cases(), ids=lambda p: p.split("/")[-1])
def test_clustering_hand_worked(nrd, path):
    hier, tags, params, expect = load_case(path)
    ctx = ctx_for(nrd, hier)
    got = ctx.regrid_boxes(dev(tags), params.get("tag_bits", 1), params["buffer"],
                           params["efficiency"], params["min_side"], params["max_side"],
                           params["max_levels"])
    assert as_lists(got) == expect


@pytest.mark.parametrize("seed", range(6))
def test_clustering_matches_oracle_random(nrd, seed):
    rng = np.random.default_rng(seed)
    n0 = [(12, 12, 12), (16, 8, 12), (10, 14, 6)][seed % 3]
    h = random_hierarchy(rng, n0, 3, count=3, side_lo=2, side_hi=5)
    tags = np.zeros(h.ncells, np.uint8)
    tags[rng.random(h.ncells) < 0.05] = 1
    tags[rng.random(h.ncells) < 0.05] |= 4
    ctx = ctx_for(nrd, h)
    for bits, buf, eff, mn, mx, ml in [(1, 1, 0.7, 4, 16, 3), (5, 0, 0.5, 2, 8, 4),
                                       (4, 2, 0.9, 2, 32, 2)]:
        got = ctx.regrid_boxes(dev(tags), bits, buf, eff, mn, mx, ml)
        exp = R.regrid_boxes(h, tags, tag_bits=bits, buffer=buf, efficiency=eff, min_side=mn,
                             max_side=mx, max_levels=ml)
        assert as_lists(got) == as_lists(exp), (bits, buf, eff, mn, mx, ml)


def test_clustering_from_device_tags(nrd):
    """Tags of the Marshak front computed on the device (nrd_tag) and in the
    oracle give the same tags and the same boxes."""
    h = W.tiny_amr(8)
    z = W.material_from_cubes(h, [((2, 2, 2), 3, 10.0)])
    u = W.front_state(h, seed=4, noise=0.0, front=0.4, width=0.1)
    ctx = ctx_for(nrd, h, z)
    t_gpu = ctx.tag(dev(u), 0.5, 0.5, float("inf"))
    o = Oracle(h, z)
    t_orc = o.tag(u, 0.5, 0.5, np.inf)
    assert np.array_equal(t_gpu.cpu().numpy(), t_orc)
    got = ctx.regrid_boxes(t_gpu, 3, 1, 0.7, 4, 16, 3)
    exp = R.regrid_boxes(h, t_orc, tag_bits=3, buffer=1, efficiency=0.7, min_side=4,
                         max_side=16, max_levels=3)
    assert as_lists(got) == as_lists(exp)
    assert len(got) >= 2


def test_regrid_errors(nrd):
    h = W.uniform(8)
    ctx = ctx_for(nrd, h)
    tags = dev(np.ones(h.ncells, np.uint8))
    with pytest.raises(nrd.NrdError):
        ctx.regrid_boxes(tags, 1, 1, 0.7, 3, 16, 2)          # odd min_side
    with pytest.raises(nrd.NrdError):
        ctx.regrid_boxes(tags, 1, 1, 1.5, 4, 16, 2)          # efficiency > 1
    with pytest.raises(nrd.NrdError):
        ctx.regrid_boxes(tags, 1, 1, 0.7, 2, 4, 3, max_boxes=1)
    other = ctx_for(nrd, W.uniform(6))
    with pytest.raises(nrd.NrdError):
        ctx.transfer_to(other, dev(np.ones(2 * h.ncells)))   # different base grids


@pytest.mark.parametrize("seed", range(4))
def test_transfer_matches_oracle(nrd, seed):
    rng = np.random.default_rng(seed)
    n0 = [(8, 8, 8), (10, 6, 8)][seed % 2]
    a = random_hierarchy(rng, n0, 3)
    b = random_hierarchy(rng, n0, 3)
    ua = np.concatenate([rng.uniform(0.1, 2.0, a.ncells), rng.uniform(0.5, 1.5, a.ncells)])
    ub = np.concatenate([rng.uniform(0.1, 2.0, a.ncells), rng.uniform(0.5, 1.5, a.ncells)])
    ca, cb = ctx_for(nrd, a), ctx_for(nrd, b)
    out = ca.transfer_to(cb, dev(np.stack([ua, ub]))).cpu().numpy()
    for k, u in enumerate((ua, ub)):
        exp = R.transfer(a, b, u)
        assert np.abs(out[k] - exp).max() <= 1e-14 * np.abs(exp).max()
    # the source is not modified by the composite step
    src = dev(ua)
    ca.transfer_to(cb, src)
    assert np.array_equal(src.cpu().numpy(), ua)


def test_transfer_full_size_conservation(nrd):
    """The benchmark hierarchy (64^3 base + Marshak band) moved to a hierarchy
    clustered from its own tags: leaf integrals of E and T conserved, the
    range kept, and sampled cells equal to the oracle's definition."""
    h, z = W.config_amr2(64, seed=0)
    u = W.front_state(h, seed=3, noise=0.0, front=0.2, width=0.05)
    ctx = ctx_for(nrd, h, z)
    tags = ctx.tag(dev(u), 0.05, 0.05, float("inf"))
    lev = ctx.regrid_boxes(tags, 3, 1, 0.7, 8, 32, 3)
    assert len(lev) >= 2
    nh = W.Hierarchy(n0=h.n0, levels=as_lists(lev))
    cn = ctx_for(nrd, nh, W.material_from_cubes(nh, []))
    v = ctx.transfer_to(cn, dev(u)).cpu().numpy()

    def vols(hh):
        L = hh.cell_ijk()[0]
        return np.array([1.0 / np.prod(hh.level_n(l)) for l in range(hh.nlevels)])[L]

    la, lb = ~h.covered_mask(), ~nh.covered_mask()
    Va, Vb = vols(h), vols(nh)
    for f in range(2):
        ua = u[f * h.ncells:(f + 1) * h.ncells]
        vb = v[f * nh.ncells:(f + 1) * nh.ncells]
        assert abs(np.sum((Va * ua)[la]) - np.sum((Vb * vb)[lb])) <= 1e-13 * np.sum(Va * ua)
        assert vb.min() >= ua[la].min() * (1 - 1e-15)
        assert vb.max() <= ua[la].max() * (1 + 1e-15)
    # sampled cells of the new level 1 against the reconstruction written out
    Lb, Ib, Jb, Kb = nh.cell_ijk()
    rng = np.random.default_rng(0)
    Lc, Ic, Jc, Kc = h.cell_ijk()
    # composite values of the old hierarchy by the paper's definition (mean of
    # the 8 children), vectorised over the base level
    E = u[:h.ncells]
    fine = np.full(h.level_n(1), np.nan)
    s1 = Lc == 1
    fine[Ic[s1], Jc[s1], Kc[s1]] = E[s1]
    base = np.full(h.level_n(0), np.nan)
    s0 = Lc == 0
    base[Ic[s0], Jc[s0], Kc[s0]] = E[s0]
    mean = fine.reshape(64, 2, 64, 2, 64, 2).mean(axis=(1, 3, 5))
    base = np.where(np.isnan(mean), base, mean)
    Lv = np.full(h.level_n(1), np.nan)
    Lv[Ic[s1], Jc[s1], Kc[s1]] = E[s1]
    for c in rng.choice(np.nonzero(Lb == 1)[0], 300, replace=False):
        q = (Ib[c], Jb[c], Kb[c])
        if not np.isnan(Lv[q]):
            assert v[c] == Lv[q]
            continue
        cq = tuple(x // 2 for x in q)
        uc = base[cq]
        val = uc
        for d in range(3):
            m = list(cq); m[d] -= 1
            p = list(cq); p[d] += 1
            if m[d] < 0 or p[d] >= 64:
                continue
            a1, b1 = uc - base[tuple(m)], base[tuple(p)] - uc
            s = 0.0 if a1 * b1 <= 0 else (a1 if abs(a1) < abs(b1) else b1)
            val += s * ((q[d] - 2 * cq[d]) + 0.5 - 1.0) / 2.0
        assert abs(v[c] - val) <= 1e-14 * abs(val)


def test_warm_restart_matches_oracle(nrd):
    """One regrid cycle on both sides: a BE step, tags, clustering, transfer of
    the solution and its history, and the re-solve of the step on the new
    hierarchy (Sec. 5 warm restart)."""
    h = W.tiny_amr(8)
    cubes = [((2, 2, 2), 3, 10.0)]
    z = W.material_from_cubes(h, cubes)
    kw = dict(pc_precision=0, nmg=2, jv_mode=nrd.JV_ANALYTIC, rtol=1e-10)
    ctx = ctx_for(nrd, h, z, **kw)
    o = Oracle(h, z)
    o.set_solver(nmg=2, jv_mode=O_AN, rtol=1e-10)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.3, width=0.08)
    dt = 2e-3
    u = dev(u0)
    st = ctx.step(u, dev(u0), None, dt)
    uo, sto = o.newton(u0.copy(), u0.copy(), 1.0, dt)
    assert st["status"] == 0 and sto["status"] == 0
    ug = u.cpu().numpy()
    # the tags and boxes are computed from the oracle's state on both sides,
    # so that no threshold decision rests on the last Newton digits
    tags_o = o.tag(uo, 0.3, 0.3, np.inf)
    t_dev = ctx.tag(dev(uo), 0.3, 0.3, float("inf"))
    assert np.array_equal(t_dev.cpu().numpy(), tags_o)
    lev = ctx.regrid_boxes(t_dev, 3, 1, 0.7, 4, 16, 3)
    lev_o = R.regrid_boxes(h, tags_o, tag_bits=3, buffer=1, efficiency=0.7, min_side=4,
                           max_side=16, max_levels=3)
    assert as_lists(lev) == as_lists(lev_o)
    nh = W.Hierarchy(n0=h.n0, levels=as_lists(lev), bc_type=h.bc_type, bc_R=h.bc_R)
    zn = W.material_from_cubes(nh, cubes)
    cn = ctx_for(nrd, nh, zn, **kw)
    moved = ctx.transfer_to(cn, torch.stack([u, dev(u0)]))
    un_o = R.transfer(h, nh, uo)
    hist_o = R.transfer(h, nh, u0)
    m = moved.cpu().numpy()
    assert np.abs(m[1] - hist_o).max() <= 1e-14 * np.abs(hist_o).max()
    assert per_cell_rel(m[0], un_o, ~nh.covered_mask()) <= 1e-8
    # re-solve the step on the new hierarchy from the transferred solution
    u2 = moved[0].clone().contiguous()
    st2 = cn.step(u2, moved[1].contiguous(), None, dt)
    on = Oracle(nh, zn)
    on.set_solver(nmg=2, jv_mode=O_AN, rtol=1e-10)
    u2o, st2o = on.newton(un_o.copy(), hist_o.copy(), 1.0, dt)
    assert st2["status"] == 0 and st2o["status"] == 0
    rel = per_cell_rel(u2.cpu().numpy(), u2o, ~nh.covered_mask())
    assert rel <= 1e-8, rel
    # the transfer left a residual jump that the re-solve removed
    assert st2["fnorm0"] > st2["fnorm"]


def test_dynamic_amr_marshak_run(nrd):
    """The dynamic-AMR Marshak run of Sec. 6 at reduced size: three z = 10
    blocks, R = 1 at x = 0 and R = 0 at x = 1, regridding every 4 steps with
    warm restarts, adaptive PC.4.7 steps.  The fine levels follow the front,
    E and T stay positive, and every re-solve converges."""
    from paper_1302_6303_gb300.amr import DynamicAmr, RegridPolicy
    n0 = (16, 16, 16)
    cubes = W.paper_blocks(n0)
    bc_type = [1, 1, 0, 0, 0, 0]
    bc_R = [1.0, 0.0, 0, 0, 0, 0]
    h = W.Hierarchy(n0=n0, levels=[[((0, 0, 0), (15, 15, 15))]], bc_type=bc_type, bc_R=bc_R)
    pol = RegridPolicy(regrid_every=4, thr_c=0.2, thr_g=0.2, tag_bits=3, buffer=1,
                       efficiency=0.7, min_side=4, max_side=16, max_levels=3)
    run = DynamicAmr(h, lambda hh: W.material_from_cubes(hh, cubes), params=None, policy=pol,
                     eps_t=1e-2, dt_max=5e-3)
    u0 = dev(W.initial_state(h))
    u = run.run(u0, 1e-4, nsteps=24)
    assert len(run.events) >= 2
    assert run.history[-1]["nlevels"] >= 2
    E = u[:run.ctx.N].cpu().numpy()
    T = u[run.ctx.N:].cpu().numpy()
    assert E.min() > 0 and T.min() > 0
    for ev in run.events:
        assert ev.fnorm_after <= ev.fnorm_before
    # the finest level covers the front: the leaf cell with the largest
    # gradient in x lies on the finest level
    L, x, y, zc = run.hier.cell_centres()
    leaf = ~run.hier.covered_mask()
    Lmax = L[leaf].max()
    front = np.abs(E - 0.5 * E.max())[leaf].argmin()
    assert L[leaf][front] == Lmax


def test_amr2_bdf2_run_with_regrids_matches_oracle(nrd):
    """The 2-level workload at base 16^3: 20 BDF2 steps (the first backward
    Euler) of dt = 5e-4 with regridding every 5 steps (tags h|grad E|/E >
    0.1, Berger-Rigoutsos with efficiency 0.7, fine boxes of 16-32 cells, a
    one-cell buffer), each regrid followed by the warm-restart re-solve of
    the last step (reading R20), on the GPU and in the oracle, compared per
    cell after every step.  The tags are computed from the oracle's state on
    both sides, so that no threshold decision rests on the last digits of
    two converged solves; the GPU's tags and boxes must equal the oracle's."""
    n0, dt, rtol = 16, 5e-4, 1e-10
    h, cubes = W.config_amr2_cubes(n0, seed=0)
    kw = dict(pc_precision=1, jv_mode=nrd.JV_ANALYTIC, rtol=rtol)

    def pair(hh):
        zz = W.material_from_cubes(hh, cubes)
        c = ctx_for(nrd, hh, zz, **kw)
        o = Oracle(hh, zz)
        o.set_solver(nmg=auto_nmg(hh), jv_mode=O_AN, rtol=rtol)
        return c, o

    ctx, o = pair(h)
    un_o = W.initial_state(h)
    un_g = dev(un_o)
    unm1_o, unm1_g = None, None
    regrids = 0
    for n in range(20):
        if unm1_o is None:
            a0, b, dtp = 1.0, un_o.copy(), 0.0
        else:
            a0, b, dtp = 1.5, 2.0 * un_o - 0.5 * unm1_o, dt   # BDF2, equal steps
        u_g = un_g.clone()
        st = ctx.step(u_g, un_g, unm1_g, dt, dtp)
        u_o, sto = o.newton(un_o.copy(), b, a0, dt)
        assert st["status"] == 0 and sto["status"] == 0, (n, st, sto)
        rel = per_cell_rel(u_g.cpu().numpy(), u_o, o.leaf_mask())
        assert rel <= 1e-8, (n, rel)
        last = (un_o, unm1_o, un_g, unm1_g, a0, dtp, sto["fnorm0"])
        unm1_o, un_o, unm1_g, un_g = un_o, u_o, un_g, u_g
        if (n + 1) % 5 or n == 19:
            continue
        # regrid on the oracle's state
        tags_o = o.tag(un_o, np.inf, np.inf, 0.1)
        t_dev = ctx.tag(dev(un_o), float("inf"), float("inf"), 0.1)
        assert np.array_equal(t_dev.cpu().numpy(), tags_o)
        lev = as_lists(ctx.regrid_boxes(t_dev, 4, 1, 0.7, 16, 32, 2))
        lev_o = as_lists(R.regrid_boxes(h, tags_o, tag_bits=4, buffer=1, efficiency=0.7,
                                        min_side=16, max_side=32, max_levels=2))
        assert lev == lev_o
        if lev == as_lists(h.levels):
            continue
        regrids += 1
        nh = W.Hierarchy(n0=h.n0, levels=lev, bc_type=h.bc_type, bc_R=h.bc_R)
        cn, on = pair(nh)
        p_un_o, p_unm1_o, p_un_g, p_unm1_g, pa0, pdtp, f0 = last
        # transfer u_{n+1}, u_n, u_{n-1} of the last step on each side
        vec_o = [un_o, p_un_o] + ([p_unm1_o] if p_unm1_o is not None else [])
        vec_g = [un_g, p_un_g] + ([p_unm1_g] if p_unm1_g is not None else [])
        mv_o = [R.transfer(h, nh, v) for v in vec_o]
        mv_g = ctx.transfer_to(cn, torch.stack(vec_g))
        for a, b_ in zip(mv_g.cpu().numpy(), mv_o):
            assert per_cell_rel(a, b_, ~nh.covered_mask()) <= 1e-8
        # warm restart: the last step solved again on the new hierarchy from
        # the transferred solution, to the absolute residual the original
        # step reached
        atol = rtol * f0
        cn.set_params(atol=atol)
        on.set_solver(nmg=auto_nmg(nh), jv_mode=O_AN, rtol=0.0, atol=atol)
        if len(mv_o) == 3:
            b2 = 2.0 * mv_o[1] - 0.5 * mv_o[2]
        else:
            b2 = mv_o[1].copy()
        u_g = mv_g[0].clone().contiguous()
        st = cn.step(u_g, mv_g[1].contiguous(),
                     mv_g[2].contiguous() if len(mv_o) == 3 else None, dt, pdtp)
        u_o, sto = on.newton(mv_o[0].copy(), b2, pa0, dt)
        assert st["status"] == 0 and sto["status"] == 0, (n, st, sto)
        assert per_cell_rel(u_g.cpu().numpy(), u_o, on.leaf_mask()) <= 1e-8
        cn.set_params(atol=0.0)
        on.set_solver(nmg=auto_nmg(nh), jv_mode=O_AN, rtol=rtol)
        h, ctx, o = nh, cn, on
        un_o, unm1_o = u_o, mv_o[1]
        un_g, unm1_g = u_g, mv_g[1].contiguous()
    assert regrids >= 1
