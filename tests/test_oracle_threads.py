"""The oracle's threaded cell loops give bit-identical results.

The oracle runs its independent per-cell loops (residual, tangent, one
colour of a red-black pass, Jacobi sweeps, restriction, prolongation,
averaging, coefficient set-up) on several host threads for the timed CPU
baseline.  Every cell's value is the same expression in the same order on
any number of threads, and the inner products stay serial, so every output
must match the single-thread run bit for bit.
"""
import numpy as np
import pytest

from oracle.oracle import JV_ANALYTIC, Oracle, set_threads
from paper_1302_6303_gb300 import workloads as W


def _run(h, z, threads, smoother):
    set_threads(threads)
    o = Oracle(h, z)
    o.set_solver(jv_mode=JV_ANALYTIC, nu1=2, nu2=1, nmg=3, coarse_sweeps=3, rtol=1e-10)
    if smoother:
        o.set_smoother(1, 0.8)
    u = W.front_state(h, seed=3, noise=0.05)
    v = W.random_direction(h, 4)
    b = u * 0.97
    out = {"F": o.residual(u, b, 1.0, 1e-3), "J": o.jv_analytic(u, v, 1.0, 1e-3)}
    o.pc_setup(u, 1.0, 1e-3)
    out["P"] = o.pc_apply(v)
    u0 = W.front_state(h, seed=5, noise=0.0, front=0.15, width=0.05)
    un, st = o.newton(u0.copy(), u0.copy(), 1.0, 1e-3)
    out["U"] = un
    out["its"] = np.array([st["newton_its"], st["krylov_its"]])
    return out


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("name", ["single16", "tiny3", "boundary"])
def test_threads_bit_identical(name, smoother):
    if name == "single16":
        h, z = W.config_single_level(16, seed=0, ncubes=2, cube_side=4)
    elif name == "tiny3":
        h = W.tiny_amr(8, three_levels=True)
        z = W.material_from_cubes(h, [((2, 2, 2), 3, 10.0)])
    else:
        h = W.boundary_amr(8)
        z = W.material_from_cubes(h, [((1, 3, 2), 3, 10.0)])
    try:
        a = _run(h, z, 1, smoother)
        if set_threads(4) < 2:
            pytest.skip("oracle built without OpenMP")
        b = _run(h, z, 4, smoother)
    finally:
        set_threads(1)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
