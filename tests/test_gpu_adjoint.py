"""Adjoint (vector-Jacobian product) parity and gradients through implicit
steps.

* nrd_vjp against the oracle's transposed Jacobian and material sensitivity
  formed column by column (tolerance 1e-12 of sum_i |w_i J_ij|);
* the transpose identity <w, J v> = <J^T w, v> at the benchmark's full size;
* the adjoint gradient of a final-time functional with respect to z and E0
  through 40 backward-Euler steps with checkpoints every 8: at base 96^3
  against central differences (h = 1e-6) of the GPU forward map on 50 cells,
  at base 24^3 against the oracle's gradient over every cell, and on a tiny
  hierarchy against the oracle's dense transposed Jacobians.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle, JV_ANALYTIC as O_AN  # noqa: E402
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


def auto_nmg(h, cap=3):
    m = 1
    while m < cap and all(n % (1 << m) == 0 for n in h.n0):
        m += 1
    return m


SMALL = {
    "single6": lambda: W.uniform(6),
    "tiny2": lambda: W.tiny_amr(8),
    "tiny3": lambda: W.tiny_amr(8, three_levels=True),
    "boundary": lambda: W.boundary_amr(8),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_vjp_against_oracle_columns(nrd, name):
    h = SMALL[name]()
    z = W.material_from_cubes(h, [((1, 2, 2), 3, 10.0)])
    ctx = nrd.Context(nmg=auto_nmg(h))
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z))
    o = Oracle(h, z)
    u = W.front_state(h, seed=3, noise=0.1)
    b = u * 0.95
    a0, dt = 1.3, 3e-3
    w = W.random_direction(h, 5)
    ctx.linearise(dev(u), dev(b), a0, dt)
    JTw, dz = ctx.vjp(dev(w), a0, dt)
    JTo, dzo, Jab = o.vjp(u, w, a0, dt)
    err = np.abs(JTw.cpu().numpy() - JTo)
    assert np.all(err <= 1e-12 * Jab + 1e-300), (err / np.maximum(Jab, 1e-300)).max()
    # material sensitivity: scale by the largest entry (brute force gives no
    # per-entry absolute scale)
    dzg = dz.cpu().numpy()
    assert np.abs(dzg - dzo).max() <= 1e-11 * np.abs(dzo).max()


def test_transpose_identity_full_size(nrd):
    h, z = W.config_amr2(64, seed=0)
    ctx = nrd.Context(tile_x=8, tile_y=8, tile_z=8)
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z))
    u = dev(W.front_state(h, seed=1, noise=0.05))
    a0, dt = 1.0, 5e-4
    ctx.linearise(u, u, a0, dt)
    v = dev(W.random_direction(h, 2))
    w = dev(W.random_direction(h, 3))
    leaf = dev(np.concatenate([~h.covered_mask()] * 2).astype(np.float64))
    v, w = v * leaf, w * leaf
    Jv = ctx.jv(u, v, a0, dt, mode=nrd.JV_FROZEN)
    JTw, _ = ctx.vjp(w, a0, dt, want_dz=False)
    lhs = float(torch.dot(w, Jv))
    rhs = float(torch.dot(JTw, v))
    scale = float(torch.dot(w.abs(), Jv.abs()))
    assert abs(lhs - rhs) <= 1e-12 * scale


def _config5(nrd, n0, front=0.5):
    """The differentiation workload: base n0^3 + 8 fine boxes near x = 0,
    40 backward-Euler steps of dt = 2.5e-4, checkpoints every 8 steps, the
    functional the integral of E over the interior (n0/6)^3 box at the final
    time; the start has a Marshak front through that box."""
    from paper_1302_6303_gb300.adjoint import StepRunner, box_weights
    h, z, fbox = W.config_adjoint(n0, seed=0, nbox=8)
    u0 = W.front_state(h, seed=2, noise=0.0, front=front, width=0.05)
    N = h.ncells
    ctx = nrd.Context(nmg=auto_nmg(h), jv_mode=nrd.JV_ANALYTIC, pc_precision=0, rtol=1e-12,
                      atol=0.0, max_newton=30)
    ctx.set_hierarchy_from(h)
    ctx.set_material(dev(z))
    wts = box_weights(h, fbox)
    runner = StepRunner(ctx, dev(u0[N:]), 40, 2.5e-4, dev(wts), ckpt_every=8)
    return h, z, u0, wts, ctx, runner


def _gpu_gradient(runner, z, E0):
    from paper_1302_6303_gb300.adjoint import ImplicitSteps
    zt = dev(z.astype(np.float64)).requires_grad_(True)
    Et = dev(E0).requires_grad_(True)
    J = ImplicitSteps.apply(zt, Et, runner)
    J.backward()
    return float(J.detach()), zt.grad.cpu().numpy(), Et.grad.cpu().numpy()


def test_gradient_full_size_against_central_differences(nrd):
    """Base 96^3, 40 steps, checkpoints every 8: the adjoint gradient with
    respect to z and E_0 against central differences (h = 1e-6 relative) of
    the GPU forward map on 50 cells: 25 drawn from the 500 cells most
    sensitive to z, 25 from the 500 most sensitive to E_0."""
    from paper_1302_6303_gb300.adjoint import ImplicitSteps
    h, z, u0, wts, ctx, runner = _config5(nrd, 96)
    N = h.ncells
    J, gz, gE = _gpu_gradient(runner, z, u0[:N])
    leaf = ~h.covered_mask()
    cand = np.nonzero(leaf)[0]
    rng = np.random.default_rng(0)
    pick_z = rng.choice(cand[np.argsort(-np.abs(gz[cand]))[:500]], 25, replace=False)
    pick_e = rng.choice(cand[np.argsort(-np.abs(gE[cand]))[:500]], 25, replace=False)

    def J_of(zz, EE):
        with torch.no_grad():
            return float(ImplicitSteps.apply(dev(zz), dev(EE), runner))

    zf = z.astype(np.float64)
    for k in pick_z:
        zp, zm = zf.copy(), zf.copy()
        zp[k] = np.float32(z[k] * (1 + 1e-6))    # z is FP32 on the device
        zm[k] = np.float32(z[k] * (1 - 1e-6))
        fd = (J_of(zp, u0[:N]) - J_of(zm, u0[:N])) / (zp[k] - zm[k])
        assert abs(fd - gz[k]) <= 1e-5 * abs(gz).max() + 1e-4 * abs(gz[k]), (k, fd, gz[k])
    for k in pick_e:
        hk = 1e-6 * abs(u0[k])
        Ep, Em = u0[:N].copy(), u0[:N].copy()
        Ep[k] += hk
        Em[k] -= hk
        fd = (J_of(zf, Ep) - J_of(zf, Em)) / (2 * hk)
        assert abs(fd - gE[k]) <= 1e-5 * abs(gE).max() + 1e-4 * abs(gE[k]), (k, fd, gE[k])


def test_gradient_against_oracle_24(nrd):
    """The same workload at base 24^3 (the layout scaled), 40 steps,
    checkpoints every 8: the GPU's adjoint gradient against the oracle's
    (oracle Newton states, sparse forward-mode Jacobians, transposed solves)
    over every cell."""
    from oracle.gradient import be_gradient
    h, z, u0, wts, ctx, runner = _config5(nrd, 24)
    N = h.ncells
    J, gz, gE = _gpu_gradient(runner, z, u0[:N])
    o = Oracle(h, z)
    o.set_solver(nmg=auto_nmg(h), jv_mode=O_AN, rtol=1e-12, max_newton=30)
    Jo, dzo, dEo = be_gradient(o, u0, 40, 2.5e-4, wts)
    assert abs(J - Jo) <= 1e-9 * abs(Jo)
    assert np.abs(gz - dzo).max() <= 1e-7 * np.abs(dzo).max()
    assert np.abs(gE - dEo).max() <= 1e-7 * np.abs(dEo).max()


def test_gradient_against_oracle(nrd):
    """The oracle's gradient: oracle Newton states, dense Jacobians from its
    forward-mode columns, transposed solves with numpy, material
    sensitivity from its column-wise (dF/dz)^T."""
    from paper_1302_6303_gb300.adjoint import ImplicitSteps, StepRunner, box_weights
    h = W.Hierarchy((8, 8, 8), [[((0, 0, 0), (7, 7, 7))], [((0, 4, 4), (5, 9, 9))]])
    z = W.material_from_cubes(h, [((2, 1, 1), 3, 10.0)])
    N = h.ncells
    u0 = W.front_state(h, seed=2, noise=0.0, front=0.3, width=0.1)
    fbox = ((2, 2, 2), (5, 5, 5))
    wts = box_weights(h, fbox)
    nsteps, dt = 3, 1e-3
    ctx = nrd.Context(nmg=2, jv_mode=nrd.JV_ANALYTIC, pc_precision=0, rtol=1e-12, max_newton=30)
    ctx.set_hierarchy_from(h)
    runner = StepRunner(ctx, dev(u0[N:]), nsteps, dt, dev(wts), ckpt_every=2)
    zt = dev(z.astype(np.float64)).requires_grad_(True)
    E0 = dev(u0[:N]).requires_grad_(True)
    J = ImplicitSteps.apply(zt, E0, runner)
    J.backward()
    # oracle
    o = Oracle(h, z)
    o.set_solver(nmg=2, jv_mode=O_AN, rtol=1e-12, max_newton=30)
    states = [u0.copy()]
    for _ in range(nsteps):
        un = states[-1]
        u, st = o.newton(un.copy(), un.copy(), 1.0, dt)
        assert st["status"] == 0
        states.append(u)
    Jo = float(np.dot(wts, states[-1][:N]))
    assert abs(Jo - float(J.detach())) <= 1e-9 * abs(Jo)
    leaf2 = np.concatenate([~h.covered_mask()] * 2)
    idx = np.nonzero(leaf2)[0]
    g = np.zeros(2 * N)
    g[:N] = wts
    dz = np.zeros(N)
    for n in reversed(range(nsteps)):
        u = states[n + 1]
        M = np.zeros((idx.size, idx.size))
        for jj, j in enumerate(idx):
            e = np.zeros(2 * N)
            e[j] = 1.0
            M[:, jj] = o.jv_analytic(u, e, 1.0, dt)[idx]
        lam = np.zeros(2 * N)
        lam[idx] = np.linalg.solve(M.T, g[idx])
        _, dzn, _ = o.vjp(u, lam, 1.0, dt)
        dz -= dzn
        g = lam
    gz = zt.grad.cpu().numpy()
    gE = E0.grad.cpu().numpy()
    assert np.abs(gz - dz).max() <= 1e-7 * np.abs(dz).max()
    assert np.abs(gE - g[:N]).max() <= 1e-7 * np.abs(g[:N]).max()
