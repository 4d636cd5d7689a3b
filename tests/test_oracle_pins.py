"""Pins of the CPU oracle against what arXiv 1302.6303 and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
from the model of Sec. 3.1 written in a different algebraic form, invariants
of the finite-volume discretisation (Sec. 3.2: conservation with flux
matching, zero flux at equilibrium), exactness of linear coarse-fine
interpolation (Sec. 3.2.1), brute-force Jacobians, eigenvalues of the
textbook 7-point operator, convergence of FAC (Algorithm 1) to a direct solve,
and second-order convergence on a manufactured solution.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, JV_ANALYTIC, JV_FD, LIM_PAPER_LITERAL, LIM_WILSON
from paper_1302_6303_gb300 import workloads as W


def vols(h):
    L, _, _, _ = h.cell_ijk()
    return np.array([1.0 / np.prod(h.level_n(l)) for l in range(h.nlevels)])[L]


def leaf_sum(o, h, x):
    m = o.leaf_mask()
    V = vols(h)
    return float(np.sum((V * x)[m]))


# ------------------------------------------------------------- equilibrium
def test_equilibrium_exact_zero_single_level():
    """Sec. 3.1: uniform E = T^4 gives zero flux and zero coupling."""
    h = W.all_neumann(W.uniform(6))
    z = W.material_from_cubes(h, [((1, 1, 1), 2, 10.0)])
    o = Oracle(h, z)
    N = h.ncells
    u = np.concatenate([np.full(N, 0.0625), np.full(N, 0.5)])  # T^4 == E exactly
    F = o.residual(u, u.copy(), 1.0, 1e-2)
    assert np.all(F == 0.0)


@pytest.mark.parametrize("three", [False, True])
def test_equilibrium_amr(three):
    h = W.all_neumann(W.tiny_amr(8, three_levels=three))
    o = Oracle(h, W.material_from_cubes(h, [((2, 2, 2), 3, 10.0)]))
    N = h.ncells
    u = np.concatenate([np.full(N, 0.0625), np.full(N, 0.5)])
    F = o.residual(u, u.copy(), 1.0, 1e-2)
    S = o.residual_scale(u, u.copy(), 1.0, 1e-2)
    assert np.all(np.abs(F) <= 1e-14 * S)


def test_robin_equilibrium():
    """Robin data R = E/4 is satisfied by a uniform E: no boundary flux."""
    h = W.uniform(5, bc_type=[1, 1, 0, 0, 0, 0], bc_R=[0.0625 / 4, 0.0625 / 4, 0, 0, 0, 0])
    o = Oracle(h, np.ones(h.ncells, np.float32))
    N = h.ncells
    u = np.concatenate([np.full(N, 0.0625), np.full(N, 0.5)])
    F = o.residual(u, u.copy(), 1.0, 1e-2)
    assert np.abs(F).max() <= 1e-17


# ------------------------------------------------------------ conservation
HIERS = {
    "single": lambda: W.uniform(6),
    "tiny2": lambda: W.tiny_amr(8),
    "tiny3": lambda: W.tiny_amr(8, three_levels=True),
    "boundary": lambda: W.boundary_amr(8),
}


@pytest.mark.parametrize("name", list(HIERS))
def test_conservation_neumann(name):
    """Sum over leaf cells of V (F_E + F_T) equals sum of V (a0 u - b): the
    coupling cancels, interior fluxes telescope and coarse-fine fluxes match
    (Sec. 3.2.1 flux matching)."""
    h = W.all_neumann(HIERS[name]())
    z = W.material_from_cubes(h, [((1, 2, 3), 3, 10.0), ((5, 0, 4), 2, 10.0)])
    o = Oracle(h, z)
    N = h.ncells
    u = W.front_state(h, seed=4)
    rng = np.random.default_rng(5)
    b = u * (1 + 0.1 * rng.uniform(-1, 1, 2 * N))
    a0, dt = 1.5, 0.05
    F = o.residual(u, b, a0, dt)
    lhs = leaf_sum(o, h, F[:N] + F[N:])
    rhs = leaf_sum(o, h, a0 * (u[:N] + u[N:]) - b[:N] - b[N:])
    S = o.residual_scale(u, b, a0, dt)
    tol = 1e-13 * leaf_sum(o, h, S[:N] + S[N:])
    assert abs(lhs - rhs) <= tol
    # the identity is not vacuous: diffusion terms are large here
    assert leaf_sum(o, h, np.abs(F[:N] - (a0 * u[:N] - b[:N]))) > 1e3 * tol


@pytest.mark.parametrize("name", ["single", "boundary"])
def test_conservation_with_robin(name):
    """With a Robin face at x = 0 the imbalance equals dt times the boundary
    flux D_b (E_0 - E_g)/h_x through that face, D_b = 1/(3 sigma_a(T_0))
    unlimited (Sec. 3.1, boundary conditions not flux limited)."""
    h = HIERS[name]()
    z = W.material_from_cubes(h, [((0, 2, 3), 3, 10.0)])
    o = Oracle(h, z)
    N = h.ncells
    u = W.front_state(h, seed=7)
    b = u.copy()
    a0, dt = 1.0, 0.02
    F = o.residual(u, b, a0, dt)
    imb = leaf_sum(o, h, F[:N] + F[N:]) - leaf_sum(o, h, a0 * (u[:N] + u[N:]) - b[:N] - b[N:])
    gE, _, _ = o.ghosts(u)
    # boundary flux from the ghost layer of x- faces of leaf cells at i = 0
    expect = 0.0
    gi = 0
    leaf = o.leaf_mask()
    L, I, J, K = h.cell_ijk()
    index = {}
    for c in range(N):
        index[(L[c], I[c], J[c], K[c])] = c
    for (l, lo, hi, off) in h.patches():
        n = [hi[d] - lo[d] + 1 for d in range(3)]
        nx = h.level_n(l)
        hx, hy, hz = 1.0 / nx[0], 1.0 / nx[1], 1.0 / nx[2]
        # face 0 (x-) is the first block of this patch's ghosts
        for kk in range(n[2]):
            for jj in range(n[1]):
                if lo[0] == 0:
                    c = index[(l, 0, lo[1] + jj, lo[2] + kk)]
                    if leaf[c]:
                        sigma = float(z[c]) ** 3 / u[N + c] ** 3
                        Db = 1.0 / (3.0 * sigma)
                        Eg = gE[gi + jj + n[1] * kk]
                        expect += dt * hy * hz * Db * (u[c] - Eg) / hx
        gi += 2 * (n[1] * n[2] + n[0] * n[2] + n[0] * n[1])
    assert expect != 0.0
    assert abs(imb - expect) <= 1e-12 * abs(expect)


def test_robin_ghost_relation_and_neumann_copy():
    """The Robin ghost satisfies (1/2) D_b dE/dn + E_face/4 = R at the face;
    Neumann ghosts equal the interior cell (zero normal derivative)."""
    h = W.uniform((4, 3, 2), bc_type=[1, 1, 0, 0, 0, 0], bc_R=[1.0, 0.3, 0, 0, 0, 0])
    z = W.material_from_cubes(h, [((0, 0, 0), 1, 10.0)])
    o = Oracle(h, z)
    N = h.ncells
    u = W.front_state(h, seed=2)
    gE, gT, gz = o.ghosts(u)
    n = (4, 3, 2)
    hx = 1.0 / 4
    sizes = [n[1] * n[2]] * 2 + [n[0] * n[2]] * 2 + [n[0] * n[1]] * 2
    starts = np.cumsum([0] + sizes)
    for face, R in ((0, 1.0), (1, 0.3)):
        i = 0 if face == 0 else n[0] - 1
        for kk in range(n[2]):
            for jj in range(n[1]):
                c = i + n[0] * (jj + n[1] * kk)
                E0, T0 = u[c], u[N + c]
                Db = 1.0 / (3.0 * (float(z[c]) ** 3 / T0 ** 3))
                Eg = gE[starts[face] + jj + n[1] * kk]
                dEdn = (Eg - E0) / hx            # outward normal derivative
                lhs = 0.5 * Db * dEdn + 0.25 * 0.5 * (Eg + E0)
                assert abs(lhs - R) <= 1e-13 * max(1.0, abs(R))
                assert gT[starts[face] + jj + n[1] * kk] == T0
    # Neumann y faces: ghost = interior
    for kk in range(n[2]):
        for ii in range(n[0]):
            c = ii + n[0] * (0 + n[1] * kk)
            assert gE[starts[2] + kk + n[2] * ii] == u[c]  # y face: z fastest, then x


# ------------------------------------------------ closed forms of the model
def _two_cell(limiter, za, zb):
    h = W.all_neumann(W.uniform((2, 1, 1)))
    z = np.array([za, zb], np.float32)
    o = Oracle(h, z, limiter=limiter)
    u = np.array([0.3, 0.05, 0.7, 0.45])  # E_a, E_b, T_a, T_b
    b = np.array([0.1, 0.2, 0.3, 0.4])
    a0, dt = 1.3, 0.07
    return o.residual(u, b, a0, dt), u, b, a0, dt


@pytest.mark.parametrize("limiter", [LIM_WILSON, LIM_PAPER_LITERAL])
@pytest.mark.parametrize("zz", [(1.0, 1.0), (1.0, 10.0)])
def test_two_cell_closed_form(limiter, zz):
    """Face D_E from Sec. 3.1: the Wilson coefficient 1/(3 sigma + |grad E|/E)
    with sigma taken as the harmonic combination of the two cells at the face
    temperature, |grad E| = |dE|/h and E the face average; D_T = k T_f^(5/2);
    coupling sigma_a (T^4 - E) with sigma_a = z^3/T^3 per cell."""
    za, zb = zz
    F, u, b, a0, dt = _two_cell(limiter, za, zb)
    Ea, Eb, Ta, Tb = u
    h = 0.5
    Tf = 0.5 * (Ta + Tb)
    # harmonic mean of the two cells' unlimited D = 1/(3 sigma) at T_f
    Da, Db_ = 1.0 / (3 * za ** 3 / Tf ** 3), 1.0 / (3 * zb ** 3 / Tf ** 3)
    Dharm = 2 * Da * Db_ / (Da + Db_)
    grad_over_E = abs(Eb - Ea) / h / (0.5 * (Ea + Eb))
    if limiter == LIM_WILSON:
        DE = 1.0 / (1.0 / Dharm + grad_over_E)
    else:  # the printed form runs the limiter at half strength
        DE = 1.0 / (1.0 / Dharm + 0.5 * grad_over_E)
    DT = 0.01 * Tf ** 2.5
    flux_E = DE * (Eb - Ea) / h
    flux_T = DT * (Tb - Ta) / h
    cpl_a = za ** 3 / Ta ** 3 * (Ta ** 4 - Ea)
    cpl_b = zb ** 3 / Tb ** 3 * (Tb ** 4 - Eb)
    fEa, fEb = flux_E / h + cpl_a, -flux_E / h + cpl_b
    fTa, fTb = flux_T / h - cpl_a, -flux_T / h - cpl_b
    expect = np.array([a0 * Ea - b[0] - dt * fEa, a0 * Eb - b[1] - dt * fEb,
                       a0 * Ta - b[2] - dt * fTa, a0 * Tb - b[3] - dt * fTb])
    np.testing.assert_allclose(F, expect, rtol=1e-13, atol=1e-15)


def test_single_cell_ode_and_newton():
    """One cell, Neumann: the residual reduces to the coupling ODE; the Newton
    solution conserves E + T and matches scipy's fsolve of the same 2x2
    backward-Euler system written from Eqs. E_td, T_td."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    h = W.all_neumann(W.uniform(1))
    z = np.array([3.0], np.float32)
    o = Oracle(h, z)
    o.set_solver(nmg=1, coarse_sweeps=1, rtol=1e-12)
    un = np.array([0.9, 0.2])
    dt = 0.05

    def be(x):
        E, T = x
        s = 27.0 / T ** 3
        return [E - un[0] - dt * s * (T ** 4 - E), T - un[1] + dt * s * (T ** 4 - E)]

    F = o.residual(un, un.copy(), 1.0, dt)
    np.testing.assert_allclose(F, be(un), rtol=1e-14)
    u, st = o.newton(un.copy(), un.copy(), 1.0, dt)
    assert st["status"] == 0
    ref = scipy_opt.fsolve(be, un, xtol=1e-14)
    np.testing.assert_allclose(u, ref, rtol=1e-10)
    assert abs(u.sum() - un.sum()) <= 1e-14


# ---------------------------------------------------------------- Jacobian
@pytest.mark.parametrize("name", ["single4", "tiny2"])
def test_dense_jacobian_vs_central_fd(name):
    """Analytic Jv columns equal brute-force central differences of F."""
    if name == "single4":
        h = W.uniform(4)
        cols = None
    else:
        h = W.tiny_amr(8)
        cols = 60
    z = W.material_from_cubes(h, [((1, 1, 1), 2, 10.0)])
    o = Oracle(h, z)
    N = h.ncells
    u = W.front_state(h, seed=11, noise=0.2)
    b = u.copy()
    a0, dt = 1.0, 0.01
    rng = np.random.default_rng(3)
    leaf = np.concatenate([o.leaf_mask()] * 2)
    idx = np.arange(2 * N)[leaf]
    if cols is not None:
        idx = rng.choice(idx, cols, replace=False)
    for j in idx:
        e = np.zeros(2 * N)
        e[j] = 1.0
        Ja = o.jv_analytic(u, e, a0, dt)
        step = 1e-6 * abs(u[j])
        up, um = u.copy(), u.copy()
        up[j] += step
        um[j] -= step
        Jc = (o.residual(up, b, a0, dt) - o.residual(um, b, a0, dt)) / (2 * step)
        scale = np.abs(Ja).max()
        assert np.abs(Ja - Jc).max() <= 2e-6 * scale, (j, np.abs(Ja - Jc).max(), scale)


@pytest.mark.parametrize("name", ["single", "tiny3"])
def test_fd_jv_close_to_analytic(name):
    h = HIERS[name]()
    o = Oracle(h, W.material_from_cubes(h, [((1, 1, 1), 2, 10.0)]))
    u = W.front_state(h, seed=2)
    v = W.random_direction(h, seed=3)
    v /= np.sqrt(o.dot(v, v))
    Ja = o.jv_analytic(u, v, 1.0, 1e-3)
    Jf, eps = o.jv_fd(u, v, u.copy(), 1.0, 1e-3)
    assert 1e-10 < abs(eps) < 1e-6
    assert np.abs(Ja - Jf).max() <= 1e-5 * np.abs(Ja).max()


def test_fd_eps_properties():
    """Sec. 4.1 differencing parameter: ~sqrt(eps_mach) <u,v>/||v||^2,
    scales as 1/c under v -> c v (both branches), keeps u + eps v > 0."""
    h = W.uniform(4)
    o = Oracle(h, np.ones(h.ncells, np.float32))
    u = W.front_state(h, seed=1)
    rng = np.random.default_rng(0)
    v = rng.uniform(0.1, 1.0, u.size)             # <u,v> > u_min ||v||_1 branch
    e1 = o.fd_eps(u, v)
    assert abs(o.fd_eps(u, 4.0 * v) - e1 / 4.0) <= 1e-15 * abs(e1)
    assert 1e-9 < e1 < 1e-6
    # second branch: <u,v> ~ 0
    v2 = rng.standard_normal(u.size)
    v2 -= o.dot(u, v2) / o.dot(u, u) * u
    e2 = o.fd_eps(u, v2)
    assert abs(o.fd_eps(u, 8.0 * v2) - e2 / 8.0) <= 1e-12 * abs(e2)
    assert abs(e2) < 1e-8 * 1e-3 * 10
    # positivity halving: one huge negative component
    v3 = v.copy()
    v3[5] = -1e9
    e3 = o.fd_eps(u, v3)
    assert np.all(u + e3 * v3 > 0)


# --------------------------------------------------------- P1 operators
def _setup_pc(h, seed=4, a0=1.0, dt=0.05, nmg=2, **kw):
    z = W.material_from_cubes(h, [((1, 2, 1), 2, 10.0)])
    o = Oracle(h, z)
    o.set_solver(nmg=nmg, **kw)
    u = W.front_state(h, seed=seed, noise=0.1)
    o.pc_setup(u, a0, dt)
    return o, u


@pytest.mark.parametrize("fld", [0, 1])
def test_linop_symmetry_single_level(fld):
    """The frozen diffusion block I - beta div D grad is symmetric in the
    volume-weighted inner product on a single level (Robin included)."""
    h = W.uniform(6)
    o, _ = _setup_pc(h)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(h.ncells), rng.standard_normal(h.ncells)
    a = np.dot(x, o.comp_apply(fld, y))
    b = np.dot(o.comp_apply(fld, x), y)
    assert abs(a - b) <= 1e-13 * np.sqrt(np.dot(x, x) * np.dot(y, y)) * 50


@pytest.mark.parametrize("fld", [0, 1])
def test_linop_fourier_eigenvalues(fld):
    """Uniform state, all Neumann: D is constant and the block is the
    textbook 7-point operator; Neumann cosine modes are eigenvectors with
    eigenvalue 1 + beta D sum_d (4/h_d^2) sin^2(pi m_d / (2 n_d))."""
    n = (6, 4, 5)
    h = W.all_neumann(W.uniform(n))
    o = Oracle(h, np.ones(h.ncells, np.float32))
    N = h.ncells
    T = 0.6
    u = np.concatenate([np.full(N, T ** 4), np.full(N, T)])
    dt = 0.03
    o.pc_setup(u, 1.0, dt)
    D = (T ** 3 / 3.0) if fld == 0 else 0.01 * T ** 2.5
    _, I, J, K = h.cell_ijk()
    for m in [(1, 0, 0), (2, 3, 1), (5, 1, 4)]:
        x = (np.cos(np.pi * m[0] * (I + 0.5) / n[0]) * np.cos(np.pi * m[1] * (J + 0.5) / n[1])
             * np.cos(np.pi * m[2] * (K + 0.5) / n[2]))
        lam = 1.0 + dt * D * sum(4.0 * n[d] ** 2 * np.sin(np.pi * m[d] / (2 * n[d])) ** 2
                                 for d in range(3))
        np.testing.assert_allclose(o.comp_apply(fld, x), lam * x, rtol=0, atol=1e-12 * lam)


@pytest.mark.parametrize("fld", [0, 1])
def test_linop_constant_on_amr(fld):
    """All Neumann: diffusion of a constant is zero across coarse-fine faces."""
    h = W.all_neumann(W.tiny_amr(8, three_levels=True))
    o, _ = _setup_pc(h, nmg=3)
    y = o.comp_apply(fld, np.ones(h.ncells))
    leaf = o.leaf_mask()
    assert np.abs(y[leaf] - 1.0).max() <= 1e-12


@pytest.mark.parametrize("fld", [0, 1])
@pytest.mark.parametrize("box", [((4, 4, 4), (11, 11, 7)), ((0, 4, 2), (7, 11, 9))],
                         ids=["interior", "robin_face"])
def test_level_operator_is_composite_with_zero_coarse_data(fld, box):
    """Algorithm 1's level error equation (reading R9: homogeneous coarse-fine
    ghosts) is the composite operator of Sec. 3.2.1 with the coarse data set
    to zero.  With one fine box every coarse value that a coarse-fine ghost
    interpolates is an uncovered coarse cell, so on every fine cell the level
    operator applied to x must equal the composite operator applied to x
    extended by zero on level 0: the ghost is then (1/3) x_f + (2/3) 0.  The
    fine cells next to the coarse-fine interface pin the level operator's
    coarse-fine row."""
    h = W.Hierarchy((8, 8, 8), [[((0, 0, 0), (7, 7, 7))], [box]])
    o, _ = _setup_pc(h, dt=0.02)
    L, I, J, K = h.cell_ijk()
    fine = L == 1
    rng = np.random.default_rng(11)
    x = np.zeros(h.ncells)
    x[fine] = rng.uniform(0.5, 1.5, int(fine.sum()))
    yc = o.comp_apply(fld, x)
    n1 = h.level_n(1)
    di = I[fine] + n1[0] * (J[fine] + n1[1] * K[fine])
    xd = np.zeros(int(np.prod(n1)))
    xd[di] = x[fine]
    yl = o.level_apply(fld, 1, xd)[di]
    assert np.abs(yl - yc[fine]).max() <= 1e-13 * np.abs(yc[fine]).max()
    # the coarse-fine rows carry a term of the size being pinned
    lo, hi = box
    edge = np.zeros(int(fine.sum()), dtype=bool)
    for d, idx in enumerate((I[fine], J[fine], K[fine])):
        edge |= ((idx == lo[d]) & (lo[d] > 0)) | ((idx == hi[d]) & (hi[d] < n1[d] - 1))
    assert edge.any()
    assert np.abs(yl[edge] - x[fine][edge]).max() > 1e-3


def test_cf_ghost_linear_exact():
    """Linear coarse-fine interpolation (Sec. 3.2.1) reproduces linear fields
    exactly at fine ghost centres; sibling ghosts are exact cell values."""
    h = W.tiny_amr(8, three_levels=True)
    o = Oracle(h, np.ones(h.ncells, np.float32))
    L, x, y, zc = h.cell_centres()
    lin = lambda X, Y, Z: 1.0 + 0.1 * X + 0.2 * Y + 0.3 * Z
    E = lin(x, y, zc)
    u = np.concatenate([E, np.full(h.ncells, 0.5)])
    u[: h.ncells] = o.average_down(u[: h.ncells].copy())  # covered = mean of children
    gE, _, _ = o.ghosts(u)
    gi = 0
    checked = 0
    for (l, lo, hi, off) in h.patches():
        if l == 0:
            gi += 6 * 64
            continue
        nl = h.level_n(l)
        n = [hi[d] - lo[d] + 1 for d in range(3)]
        for face in range(6):
            d, s = face // 2, (1 if face % 2 else -1)
            t1, t2 = (d + 1) % 3, (d + 2) % 3
            for b2 in range(lo[t2], hi[t2] + 1):
                for b1 in range(lo[t1], hi[t1] + 1):
                    c = [0, 0, 0]
                    c[d] = (lo[d] - 1) if s < 0 else (hi[d] + 1)
                    c[t1], c[t2] = b1, b2
                    X = [(c[a] + 0.5) / nl[a] for a in range(3)]
                    assert abs(gE[gi] - lin(*X)) <= 1e-14, (l, face, c)
                    gi += 1
                    checked += 1
    assert checked > 0


def test_gmg_textbook_convergence():
    """One V(2,2) cycle of the GMG on a constant-coefficient Neumann problem
    contracts the error by a textbook factor (< 0.15) when the coarsest grid
    (one cell, where the operator is the identity) is solved exactly."""
    h = W.all_neumann(W.uniform(16))
    o = Oracle(h, np.ones(h.ncells, np.float32))
    o.set_solver(nmg=5, nu1=2, nu2=2)
    N = h.ncells
    T = 0.9
    u = np.concatenate([np.full(N, T ** 4), np.full(N, T)])
    o.pc_setup(u, 1.0, 5.0)  # strongly diffusion dominated
    rng = np.random.default_rng(0)
    f = rng.standard_normal(N)
    x = np.zeros(N)
    rn = []
    for _ in range(6):
        r = f - o.comp_apply(0, x)
        rn.append(np.linalg.norm(r))
        x += o.gmg(0, r)
    rates = np.array(rn[1:]) / np.array(rn[:-1])
    assert rates[-1] < 0.15, rates


def test_fac_single_level_equals_gmg():
    h = W.uniform(8)
    o, _ = _setup_pc(h, nmg=3)
    rng = np.random.default_rng(2)
    f = rng.standard_normal(h.ncells)
    for fld in (0, 1):
        np.testing.assert_array_equal(o.fac(fld, f), o.gmg(fld, f))


@pytest.mark.parametrize("three", [False, True])
@pytest.mark.parametrize("fld", [0, 1])
def test_fac_converges_to_direct_solve(three, fld):
    """Iterating FAC V-cycles (Algorithm 1) converges, at a multigrid rate,
    to the dense direct solution of the composite operator L^c."""
    h = W.tiny_amr(8, three_levels=three)
    o, _ = _setup_pc(h, nmg=3, dt=0.2)
    leaf = o.leaf_mask()
    idx = np.nonzero(leaf)[0]
    N = h.ncells
    A = np.zeros((idx.size, idx.size))
    for jj, j in enumerate(idx):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, jj] = o.comp_apply(fld, e)[idx]
    rng = np.random.default_rng(7)
    f = np.zeros(N)
    f[idx] = rng.standard_normal(idx.size)
    xd = np.linalg.solve(A, f[idx])
    x = np.zeros(N)
    errs = []
    for _ in range(12):
        r = f - o.comp_apply(fld, x)
        r[~leaf] = 0.0
        x += o.fac(fld, r)
        errs.append(np.abs(x[idx] - xd).max())
    assert errs[-1] <= 1e-10 * np.abs(xd).max()
    assert errs[3] / errs[2] < 0.5


@pytest.mark.parametrize("fld", [0, 1])
def test_jacobi_sweeps_match_dense_formula(fld):
    """The damped point Jacobi smoother (Sec. 4.3 names it beside red-black
    Gauss-Seidel) takes, from e = 0, e_1 = w D^-1 f and then
    e_(k+1) = e_k + w D^-1 (f - A e_k), with A the dense single-level
    operator (Robin and Neumann faces) and D its diagonal: the smoothing-only
    coarsest level (one GMG level) with 1 and 3 sweeps."""
    h = W.uniform(5)
    N = h.ncells
    rng = np.random.default_rng(3)
    f = rng.standard_normal(N)
    w = 0.7
    for sweeps in (1, 3):
        o, _ = _setup_pc(h, nmg=1, coarse_sweeps=sweeps)
        o.set_smoother(1, w)
        A = np.zeros((N, N))
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            A[:, j] = o.comp_apply(fld, e)
        D = np.diag(A)
        x = w * f / D
        for _ in range(sweeps - 1):
            x = x + w * (f - A @ x) / D
        y = o.gmg(fld, f)
        assert np.abs(y - x).max() <= 1e-13 * np.abs(x).max()


@pytest.mark.parametrize("fld", [0, 1])
def test_fac_with_jacobi_converges_to_direct_solve(fld):
    """FAC (Algorithm 1) with the damped Jacobi smoother on every level and
    the coarse GMG grids still converges to the dense direct solution of the
    composite operator."""
    h = W.tiny_amr(8)
    o, _ = _setup_pc(h, nmg=3, dt=0.2)
    o.set_smoother(1, 6.0 / 7.0)
    leaf = o.leaf_mask()
    idx = np.nonzero(leaf)[0]
    N = h.ncells
    A = np.zeros((idx.size, idx.size))
    for jj, j in enumerate(idx):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, jj] = o.comp_apply(fld, e)[idx]
    rng = np.random.default_rng(8)
    f = np.zeros(N)
    f[idx] = rng.standard_normal(idx.size)
    xd = np.linalg.solve(A, f[idx])
    x = np.zeros(N)
    errs = []
    for _ in range(40):
        r = f - o.comp_apply(fld, x)
        r[~leaf] = 0.0
        x += o.fac(fld, r)
        errs.append(np.abs(x[idx] - xd).max())
    assert errs[-1] <= 1e-10 * np.abs(xd).max()
    assert errs[5] / errs[4] < 0.8


@pytest.mark.parametrize("fld", [0, 1])
def test_xline_block_gs_matches_dense_block_gs(fld):
    """Block Gauss-Seidel (Sec. 4.3; reading R26: x-line blocks of a box
    level solved exactly, lines coloured by j + k, red first in
    pre-smoothing) against the same iteration written densely: A the
    single-level operator from its columns, each block's rows solved with
    numpy against the current values outside the block.  One and three
    sweeps on the smoothing-only coarsest level (one GMG level), and a
    single-line box, where one sweep is the exact solve."""
    for n, sweeps in (((6, 4, 4), 1), ((6, 4, 4), 3), ((9, 1, 1), 1)):
        h = W.uniform(n)
        N = h.ncells
        o, _ = _setup_pc(h, nmg=1, coarse_sweeps=sweeps)
        o.set_smoother(2)
        A = np.zeros((N, N))
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            A[:, j] = o.comp_apply(fld, e)
        f = np.random.default_rng(4).standard_normal(N)
        L, I, J, K = h.cell_ijk()
        x = np.zeros(N)
        for _ in range(sweeps):
            for colour in (0, 1):
                for k in range(n[2]):
                    for j in range(n[1]):
                        if (j + k) % 2 != colour:
                            continue
                        blk = np.nonzero((J == j) & (K == k))[0]
                        rest = np.setdiff1d(np.arange(N), blk)
                        rhs = f[blk] - A[np.ix_(blk, rest)] @ x[rest]
                        x[blk] = np.linalg.solve(A[np.ix_(blk, blk)], rhs)
        y = o.gmg(fld, f)
        assert np.abs(y - x).max() <= 1e-12 * np.abs(x).max()
        if n[1] == 1:
            assert np.abs(A @ y - f).max() <= 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("fld", [0, 1])
def test_fac_with_block_gs_converges_to_direct_solve(fld):
    """FAC with x-line block Gauss-Seidel on the GMG box levels (point
    red-black sweeps on the patch levels) converges to the dense direct
    solution of the composite operator."""
    h = W.tiny_amr(8)
    o, _ = _setup_pc(h, nmg=3, dt=0.2)
    o.set_smoother(2)
    leaf = o.leaf_mask()
    idx = np.nonzero(leaf)[0]
    N = h.ncells
    A = np.zeros((idx.size, idx.size))
    for jj, j in enumerate(idx):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, jj] = o.comp_apply(fld, e)[idx]
    f = np.zeros(N)
    f[idx] = np.random.default_rng(8).standard_normal(idx.size)
    xd = np.linalg.solve(A, f[idx])
    x = np.zeros(N)
    errs = []
    for _ in range(40):
        r = f - o.comp_apply(fld, x)
        r[~leaf] = 0.0
        x += o.fac(fld, r)
        errs.append(np.abs(x[idx] - xd).max())
    assert errs[-1] <= 1e-10 * np.abs(xd).max()
    assert errs[5] / errs[4] < 0.8


def test_p2_solve_matches_printed_matrix():
    """y = P^{-1} w = P2^{-1} P1^{-1} w with P2 as printed in Sec. 4.2."""
    h = W.uniform(4)
    o, u = _setup_pc(h, nmg=2, dt=0.1)
    N = h.ncells
    rng = np.random.default_rng(9)
    w = rng.standard_normal(2 * N)
    y = o.pc_apply(w)
    zE, zT = o.fac(0, w[:N]), o.fac(1, w[N:])
    T = u[N:]
    zc = W.material_from_cubes(h, [((1, 2, 1), 2, 10.0)]).astype(np.float64)
    sig = zc ** 3 / T ** 3
    beta = 0.1
    yE, yT = y[:N], y[N:]
    r1 = (1 + sig * beta) * yE - sig * beta * T ** 3 * yT
    r2 = -sig * beta * yE + (1 + sig * beta * T ** 3) * yT
    np.testing.assert_allclose(r1, zE, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r2, zT, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ Newton
@pytest.mark.parametrize("name", ["single", "tiny2"])
def test_newton_solution_independent_of_solver_settings(name):
    h = {"single": lambda: W.uniform(8), "tiny2": lambda: W.tiny_amr(8)}[name]()
    z = W.material_from_cubes(h, [((1, 2, 1), 3, 10.0)])
    u0 = W.front_state(h, seed=5, noise=0.02)
    sols = []
    for kw in [dict(nu1=2, nu2=2, nmg=3, jv_mode=JV_FD),
               dict(nu1=1, nu2=0, nmg=1, jv_mode=JV_FD),
               dict(nu1=2, nu2=2, nmg=3, jv_mode=JV_ANALYTIC)]:
        o = Oracle(h, z)
        o.set_solver(rtol=1e-10, **kw)
        u, st = o.newton(u0.copy(), u0.copy(), 1.0, 2e-3)
        assert st["status"] == 0 and st["fnorm"] <= 1e-10 * st["fnorm0"]
        leaf = np.concatenate([o.leaf_mask()] * 2)
        sols.append(u[leaf])
    for s in sols[1:]:
        np.testing.assert_allclose(s, sols[0], rtol=1e-8)


# ------------------------------------------------- manufactured solution
def _mms_funcs():
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x", real=True)
    E = sp.Rational(1, 2) + sp.Rational(1, 4) * sp.cos(sp.pi * x)
    T = sp.Rational(4, 5) + sp.Rational(1, 10) * sp.cos(sp.pi * x)
    sigma = 1 / T ** 3                                   # z = 1
    dE = sp.diff(E, x)
    # Wilson limiter D_E = 1/(3 sigma + |grad E|/E) with |grad E| = |E_x|
    DE = 1 / (3 * sigma + sp.Abs(dE) / E)
    DT = sp.Rational(1, 100) * T ** sp.Rational(5, 2)
    cpl = sigma * (T ** 4 - E)
    fE = sp.diff(DE * dE, x) + cpl
    fT = sp.diff(DT * sp.diff(T, x), x) - cpl
    lam = lambda ex: sp.lambdify(x, ex, "numpy")
    return lam(E), lam(T), lam(fE), lam(fT)


def _mms_error(h, funcs, dt=0.05):
    Ef, Tf, fEf, fTf = funcs
    o = Oracle(h, np.ones(h.ncells, np.float32))
    o.set_solver(rtol=1e-11, nmg=1, nu1=2, nu2=2, coarse_sweeps=4, jv_mode=JV_ANALYTIC)
    L, x, y, z = h.cell_centres()
    us = np.concatenate([Ef(x), Tf(x)])
    fs = np.concatenate([fEf(x), fTf(x)])
    b = us - dt * fs                       # makes u* the exact semi-discrete step
    u, st = o.newton(1.05 * us, b, 1.0, dt)
    assert st["status"] == 0
    leaf = np.concatenate([o.leaf_mask()] * 2)
    return np.abs(u - us)[leaf].max()


def test_mms_second_order_uniform():
    """Second-order spatial accuracy (Sec. 6 accuracy study) on a smooth
    manufactured 1D profile with Neumann walls."""
    funcs = _mms_funcs()
    errs = [_mms_error(W.all_neumann(W.uniform((n, 1, 1))), funcs) for n in (16, 32, 64)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


def test_mms_amr_second_order():
    """With a refined patch (linear coarse-fine interpolation plus flux
    matching) the solution error still converges at second order, the claim
    of Sec. 3.2.1; a wrong interpolation weight drops this to first order."""
    funcs = _mms_funcs()
    errs = []
    for n in (16, 32, 64):
        lv1 = [((n // 2, 0, 0), (n + n // 2 - 1, 1, 1))]
        h = W.all_neumann(W.Hierarchy((n, 1, 1), [[((0, 0, 0), (n - 1, 0, 0))], lv1]))
        errs.append(_mms_error(h, funcs))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


# -------------------------------------------------------------- tagging
def test_tag_linear_field():
    """Sec. 5 indicators on E linear in x: curvature indicator 0 away from the
    boundary, gradient indicator h |E_x| / (0.1 max E) exactly."""
    h = W.all_neumann(W.uniform(8))
    o = Oracle(h, np.ones(h.ncells, np.float32))
    L, x, y, z = h.cell_centres()
    E = 0.2 + 0.5 * x
    u = np.concatenate([E, np.full(h.ncells, 0.5)])
    emax = E.max()
    tg = (1.0 / 8) * 0.5 / (0.1 * emax)
    _, I, J, K = h.cell_ijk()
    inner = (I > 0) & (I < 7)
    t = o.tag(u, thr_g=tg * (1 - 1e-9))
    assert np.all((t[inner] & 2) == 2)
    t = o.tag(u, thr_g=tg * (1 + 1e-9))
    assert np.all((t[inner] & 2) == 0)
    t = o.tag(u, thr_c=1e-9)
    assert np.all((t[inner] & 1) == 0)
    rel = np.sqrt((0.5 / 8) ** 2) / E
    t = o.tag(u, thr_r=0.0)
    assert np.all(t[inner] & 4)
    tr = o.tag(u, thr_r=float(rel[inner].max()) * (1 + 1e-9))
    assert np.all((tr[inner] & 4) == 0)


# ------------------------------------------------------------------ adjoint
def _tiny2():
    h = W.Hierarchy((4, 4, 4), [[((0, 0, 0), (3, 3, 3))], [((2, 2, 2), (5, 5, 5))]])
    return h


@pytest.mark.parametrize("name", ["single", "tiny2"])
def test_vjp_matches_central_differences(name):
    """(dF/du)^T w and (dF/dz)^T w equal central differences of the scalar
    phi = <w, F(u; z)> (plain sum) in every u_j and z_k."""
    h = W.uniform((3, 3, 2)) if name == "single" else _tiny2()
    z = W.material_from_cubes(h, [((1, 1, 0), 2, 10.0)]).astype(np.float64)
    o = Oracle(h)
    o.set_material_f64(z)
    N = h.ncells
    u = W.front_state(h, seed=3, noise=0.2)
    b = u * 0.9
    a0, dt = 1.1, 0.02
    w = np.random.default_rng(1).standard_normal(2 * N)
    JTw, dz, _ = o.vjp(u, w, a0, dt)
    phi = lambda uu: float(np.dot(w, o.residual(uu, b, a0, dt)))
    fd = np.empty(2 * N)
    for j in range(2 * N):
        hj = 1e-6 * abs(u[j])
        up, um = u.copy(), u.copy()
        up[j] += hj
        um[j] -= hj
        fd[j] = (phi(up) - phi(um)) / (2 * hj)
    leaf = np.concatenate([o.leaf_mask()] * 2)
    np.testing.assert_allclose(JTw[leaf], fd[leaf], rtol=0, atol=1e-6 * np.abs(fd).max())
    assert np.all(JTw[~leaf] == 0.0)
    fz = np.empty(N)
    for k in range(N):
        hk = 1e-6 * z[k]
        zp, zm = z.copy(), z.copy()
        zp[k] += hk
        zm[k] -= hk
        o.set_material_f64(zp)
        fp = phi(u)
        o.set_material_f64(zm)
        fm = phi(u)
        fz[k] = (fp - fm) / (2 * hk)
    o.set_material_f64(z)
    np.testing.assert_allclose(dz, fz, rtol=0, atol=1e-6 * np.abs(fz).max())


# ---------------------------------------------------------- step control
def _tfield(h, f):
    """a field whose every component is f(t) times a positive spatial shape"""
    L, x, y, zc = h.cell_centres()
    shape = np.concatenate([1.0 + x + 0.5 * y, 2.0 + zc])
    return lambda t: shape * f(t)


@pytest.mark.parametrize("alpha", [1.0, 0.5, 2.0])
def test_leapfrog_predictor_error_closed_form(alpha):
    """Eq. leapfrog with the exact derivative: exact for quadratics in time;
    for u = t^3 its error is -(1 + dt_{n-1}/dt_n) dt_n^3/6 u''' (Sec. 3.5)."""
    h = W.uniform(3)
    o = Oracle(h, np.ones(h.ncells, np.float32))
    tau = 0.01
    dt = alpha * tau
    for f, df, err in [(lambda t: 1 + 2 * t + 3 * t * t, lambda t: 2 + 6 * t, lambda: 0.0),
                       (lambda t: t ** 3, lambda t: 3 * t * t,
                        lambda: -(1 + tau / dt) * dt ** 3 / 6 * 6)]:
        u = _tfield(h, f)
        ud = _tfield(h, df)
        up = o.predict(u(0.0), u(-tau), ud(0.0), dt, tau)
        shape = _tfield(h, lambda t: 1.0)(0.0)
        np.testing.assert_allclose(up - u(dt), err() * shape, rtol=0, atol=1e-14 * np.abs(u(dt)).max())


@pytest.mark.parametrize("alpha", [1.0, 0.5, 2.0])
def test_bdf2_error_estimate_exact_for_cubics(alpha):
    """For u' = 3 t^2 (solution t^3) the BDF2 step from exact history, the
    derivative from the left-hand side of Eq. bdf2 and the estimate of Eq.
    bdf2le recover the true local error."""
    h = W.uniform(2)
    o = Oracle(h, np.ones(h.ncells, np.float32))
    tau = 0.02
    dt = alpha * tau
    u = _tfield(h, lambda t: t ** 3)
    un, unm1 = u(0.0), u(-tau)
    # the BDF2 step: time derivative at t_{n+1} equals f = 3 t_{n+1}^2 (the
    # derivative is affine in u_{n+1}: solve it from two evaluations)
    shape = _tfield(h, lambda t: 1.0)(0.0)
    target = 3 * dt * dt * shape
    d0 = o.time_derivative(np.zeros_like(un), un, unm1, dt, tau)
    d1 = o.time_derivative(np.ones_like(un), un, unm1, dt, tau)
    u1 = (target - d0) / (d1 - d0)
    true_err = u1 - u(dt)
    # predictor with the derivative at t_n from the previous BDF2 step's LHS is
    # not exact; use the exact derivative, as in the derivation of Eq. bdf2le
    up = o.predict(un, unm1, _tfield(h, lambda t: 3 * t * t)(0.0), dt, tau)
    est = (alpha + 1) / (3 * alpha + 2) * (u1 - up)
    np.testing.assert_allclose(est, true_err, rtol=1e-10, atol=1e-18)
    # and the scaled max norm
    m = o.lte(u1, up, alpha, eta_E=0.5, eta_T=0.25)
    N = h.ncells
    ref = max(np.max(np.abs(est[:N] / (u1[:N] + 0.5))), np.max(np.abs(est[N:] / (u1[N:] + 0.25))))
    assert abs(m - ref) <= 1e-15 * ref


# ------------------------------------------------ gradient through the steps
def test_oracle_sparse_jacobian_matches_forward_and_transposed_products():
    """The sparse forward-mode Jacobian reproduces the analytic Jv (pinned by
    the dense central-difference Jacobians above) and the transposed
    products by columns, in u and in z."""
    for h in (W.tiny_amr(8, three_levels=True), W.boundary_amr(8)):
        z = W.material_from_cubes(h, [((2, 2, 2), 3, 10.0)])
        o = Oracle(h, z)
        u = W.front_state(h, seed=3, noise=0.1)
        Ju, Jz = o.jacobian(u, 1.3, 3e-3)
        v = W.random_direction(h, 4)
        Jv = o.jv_analytic(u, v, 1.3, 3e-3)
        assert np.abs(Ju @ v - Jv).max() <= 1e-14 * np.abs(Jv).max()
        w = W.random_direction(h, 5)
        JTw, dz, _ = o.vjp(u, w, 1.3, 3e-3)
        assert np.abs(Ju.T @ w - JTw).max() <= 1e-14 * np.abs(JTw).max()
        assert np.abs(Jz.T @ w - dz).max() <= 1e-14 * np.abs(dz).max()


def test_oracle_gradient_against_central_differences():
    """The oracle's discrete adjoint through backward-Euler steps against
    central differences of its own converged forward map J(z, E_0)."""
    from oracle.gradient import be_gradient
    from paper_1302_6303_gb300.adjoint import box_weights
    h = W.Hierarchy((8, 8, 8), [[((0, 0, 0), (7, 7, 7))], [((0, 4, 4), (5, 9, 9))]])
    z = W.material_from_cubes(h, [((2, 1, 1), 3, 10.0)])
    N = h.ncells
    u0 = W.front_state(h, seed=2, noise=0.0, front=0.3, width=0.1)
    w = box_weights(h, ((2, 2, 2), (5, 5, 5)))
    nsteps, dt = 3, 1e-3

    def oracle(zz):
        o = Oracle(h, None)
        o.set_material_f64(zz)
        o.set_solver(jv_mode=JV_ANALYTIC, nmg=2, rtol=1e-13, max_newton=30)
        return o

    zz = z.astype(np.float64)
    J, dz, dE = be_gradient(oracle(zz), u0, nsteps, dt, w)

    def J_of(zv, E):
        o = oracle(zv)
        u = np.concatenate([E, u0[N:]])
        for _ in range(nsteps):
            u, st = o.newton(u.copy(), u.copy(), 1.0, dt)
            assert st["status"] == 0
        return float(np.dot(w, u[:N]))

    assert abs(J_of(zz, u0[:N]) - J) <= 1e-12 * abs(J)
    for k in np.argsort(-np.abs(dz))[:3]:
        hz = 1e-6 * zz[k]
        zp, zm = zz.copy(), zz.copy()
        zp[k] += hz
        zm[k] -= hz
        fd = (J_of(zp, u0[:N]) - J_of(zm, u0[:N])) / (2 * hz)
        assert abs(fd - dz[k]) <= 1e-6 * np.abs(dz).max(), (k, fd, dz[k])
    for k in np.argsort(-np.abs(dE))[:3]:
        he = 1e-6 * u0[k]
        Ep, Em = u0[:N].copy(), u0[:N].copy()
        Ep[k] += he
        Em[k] -= he
        fd = (J_of(zz, Ep) - J_of(zz, Em)) / (2 * he)
        assert abs(fd - dE[k]) <= 1e-6 * np.abs(dE).max(), (k, fd, dE[k])
