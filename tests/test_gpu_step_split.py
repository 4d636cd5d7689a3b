"""The implicit step in two halves (nrd_step_begin / nrd_step_end, Sec. 3.3):
the same result and statistics as nrd_step, work enqueued behind a pending
step on its stream, and the state rules while a step is pending."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1302_6303_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def nrd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(nrd, h, z, **kw):
    ctx = nrd.Context(**kw)
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z.astype(np.float32)))
    return ctx


@pytest.mark.parametrize("form", ["graph", "host"])
def test_split_step_equals_step(nrd, form):
    """BDF2 after a BE step, both halves against nrd_step: bit-identical u
    and identical iteration counts, for the device-loop (graph) form and the
    host-driven loop (FD Jv)."""
    h, z = W.config_amr2(16, seed=3, band=4, ncubes=4)
    kw = dict(jv_mode=nrd.JV_ANALYTIC, rtol=1e-10) if form == "graph" else \
        dict(jv_mode=nrd.JV_FD, rtol=1e-10)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    dt = 1e-3
    runs = []
    for split in (False, True):
        ctx = make(nrd, h, z, **kw)
        un = dev(u0)
        u1 = un.clone()
        st1 = ctx.step(u1, un, None, dt)
        u2 = u1.clone()
        if split:
            ctx.step_begin(u2, u1, un, dt, dt)
            st2 = ctx.step_end()
        else:
            st2 = ctx.step(u2, u1, un, dt, dt)
        torch.cuda.synchronize()
        runs.append((u2.cpu().numpy(), st1, st2))
    (ua, _, sa), (ub, _, sb) = runs
    assert sa["status"] == 0 and sb["status"] == 0
    assert np.array_equal(ua, ub)
    for k in ("newton_its", "krylov_its", "pc_setups"):
        assert sa[k] == sb[k], k


def test_work_behind_a_pending_step(nrd):
    """The time derivative and the indicators enqueued behind a pending step
    see its result: the same values as when called after nrd_step."""
    h, z = W.config_amr2(16, seed=3, band=4, ncubes=4)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    dt = 1e-3
    out = []
    for split in (False, True):
        ctx = make(nrd, h, z, jv_mode=nrd.JV_ANALYTIC, rtol=1e-10)
        un = dev(u0)
        u = un.clone()
        if split:
            ctx.step_begin(u, un, None, dt)
        else:
            ctx.step(u, un, None, dt)
        ud = ctx.time_derivative(u, un, None, dt)
        tg = ctx.tag(u, thr_r=0.1)
        if split:
            assert ctx.step_end()["status"] == 0
        torch.cuda.synchronize()
        out.append((ud.cpu().numpy(), tg.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_pending_step_state_rules(nrd):
    """While a step is pending: a second begin, a residual, a parameter change
    and a call on another stream return NRD_ESTATE; the step ends normally;
    an end without a pending step returns NRD_ESTATE."""
    h, z = W.config_amr2(16, seed=3, band=4, ncubes=4)
    u0 = W.front_state(h, seed=9, noise=0.0, front=0.1, width=0.05)
    ctx = make(nrd, h, z, jv_mode=nrd.JV_ANALYTIC, rtol=1e-10)
    un = dev(u0)
    u = un.clone()
    ctx.step_begin(u, un, None, 1e-3)
    with pytest.raises(nrd.NrdError) as e:
        ctx.step_begin(u, un, None, 1e-3)
    assert e.value.code == nrd.ESTATE
    with pytest.raises(nrd.NrdError) as e:
        ctx.residual(u, un, 1.0, 1e-3)
    assert e.value.code == nrd.ESTATE
    with pytest.raises(nrd.NrdError) as e:
        ctx.set_params(nu1=2)
    assert e.value.code == nrd.ESTATE
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with pytest.raises(nrd.NrdError) as e:
            ctx.tag(u, thr_r=0.1)
    assert e.value.code == nrd.ESTATE
    st = ctx.step_end()
    assert st["status"] == 0 and st["newton_its"] >= 1
    with pytest.raises(nrd.NrdError) as e:
        ctx.step_end()
    assert e.value.code == nrd.ESTATE
    # usable again
    F = ctx.residual(u, un, 1.0, 1e-3)
    assert torch.isfinite(F).all()
