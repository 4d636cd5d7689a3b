"""Time-step control (Sec. 3.4-3.5): GPU kernels against the oracle, the
controllers' defining properties, and an adaptive BDF2 run whose states the
oracle reproduces with the same step sequence."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle, JV_ANALYTIC as O_AN  # noqa: E402
from paper_1302_6303_gb300 import workloads as W  # noqa: E402
from stepcheck import per_cell_rel  # noqa: E402


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


def test_predictor_derivative_lte_parity(nrd):
    h = W.tiny_amr(8)
    z = W.material_from_cubes(h, [((1, 1, 1), 3, 10.0)])
    ctx = nrd.Context(nmg=2)
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z))
    o = Oracle(h, z)
    rng = np.random.default_rng(0)
    u1 = W.front_state(h, seed=1)
    u0 = u1 * (1 + 0.01 * rng.uniform(-1, 1, u1.size))
    um = u0 * (1 + 0.01 * rng.uniform(-1, 1, u1.size))
    dt, dtp = 1e-3, 7e-4
    for prev in (None, um):
        d = ctx.time_derivative(dev(u1), dev(u0), None if prev is None else dev(prev), dt,
                                dtp).cpu().numpy()
        do = o.time_derivative(u1, u0, prev, dt, dtp)
        np.testing.assert_allclose(d, do, rtol=1e-13, atol=1e-13 * np.abs(do).max())
    ud = o.time_derivative(u0, um, None, dtp)
    up = ctx.predict(dev(u0), dev(um), dev(ud), dt, dtp).cpu().numpy()
    upo = o.predict(u0, um, ud, dt, dtp)
    np.testing.assert_allclose(up, upo, rtol=1e-13, atol=1e-15)
    e = ctx.lte(dev(u1), dev(upo), dt / dtp, 1e-5, 1e-3)
    eo = o.lte(u1, upo, dt / dtp, 1e-5, 1e-3)
    assert abs(e - eo) <= 1e-13 * eo


def test_controllers(nrd):
    # EPS: error at the target keeps dt; 8x the error halves it (k = 3)
    assert abs(nrd.dt_control(nrd.DT_EPS, 1e-3, 1e-3, 0, 0.1, 0.1) - 0.1) < 1e-15
    assert abs(nrd.dt_control(nrd.DT_EPS, 1e-3, 8e-3, 0, 0.1, 0.1) - 0.05) < 1e-15
    # PC.4.7: at the target with a steady error the step ratio is kept
    assert abs(nrd.dt_control(nrd.DT_PC47, 1e-3, 1e-3, 1e-3, 0.2, 0.1) - 0.4) < 1e-14
    # growing error shrinks the step more than the integral term alone
    a = nrd.dt_control(nrd.DT_PC47, 1e-3, 2e-3, 1e-3, 0.1, 0.1)
    b = nrd.dt_control(nrd.DT_PC47, 1e-3, 2e-3, 2e-3, 0.1, 0.1)
    assert a < b < 0.1
    with pytest.raises(nrd.NrdError):
        nrd.dt_control(nrd.DT_PC47, 1e-3, 0.0, 1e-3, 0.1, 0.1)


def test_adaptive_run_matches_oracle_steps(nrd):
    from paper_1302_6303_gb300.stepper import Integrator
    h, z = W.config_single_level(16, seed=2, ncubes=2, cube_side=4)
    ctx = nrd.Context(nmg=3, jv_mode=nrd.JV_ANALYTIC, pc_precision=0, rtol=1e-11)
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z))
    u0 = W.front_state(h, seed=0, noise=0.0, front=0.1, width=0.05)
    integ = Integrator(ctx, eps_t=1e-3)
    u = integ.run(dev(u0), 2e-4, nsteps=6)
    hist = integ.history
    assert all(r["status"] == 0 for r in hist)
    dts = [r["dt"] for r in hist]
    assert len(set(round(d, 15) for d in dts)) > 1      # the controller acted
    # the oracle with the same step sequence (BE then variable BDF2)
    o = Oracle(h, z)
    o.set_solver(nmg=3, jv_mode=O_AN, rtol=1e-11)
    un, unm1, dtp = u0.copy(), None, None
    for dt in dts:
        if unm1 is None:
            b, a0 = un.copy(), 1.0
        else:
            al = dt / dtp
            a0 = (1 + 2 * al) / (1 + al)
            b = (1 + al) * un - al * al / (1 + al) * unm1
        u1, st = o.newton(un.copy(), b, a0, dt)
        assert st["status"] == 0
        unm1, un, dtp = un, u1, dt
    rel = per_cell_rel(u.cpu().numpy(), un, o.leaf_mask())
    assert rel <= 1e-8, rel
