"""The oracle's gradient through implicit backward-Euler steps.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone.  It shares no code
with the CUDA library.

J = sum_c w_c E_c(t_final) after `nsteps` backward-Euler steps (Sec. 3.3 with
a0 = 1, b = u_n) from u_0 = (E_0, T_0), each solved to convergence by the
oracle's Newton.  For a step F(u_{n+1}; u_n, z) = u_{n+1} - u_n - dt f(u_{n+1};
z) = 0 the discrete adjoint is the plain chain rule:
  lambda_n solves (dF/du_{n+1})^T lambda_n = g_{n+1}   (on the leaf unknowns),
  g_n = -(dF/du_n)^T lambda_n = lambda_n,
  dJ/dz -= (dF/dz)^T lambda_n,
with g_nsteps = dJ/du(t_final) = (w, 0) and dJ/dE_0 = the E part of g_0.  The
Jacobians are the oracle's sparse forward-mode ones (Oracle.jacobian); the
transposed systems are solved by scipy's GMRES with the diagonal as
preconditioner to a relative residual of 1e-14, the true residual checked.
"""
from __future__ import annotations

import numpy as np


def be_gradient(o, u0, nsteps, dt, weights):
    """(J, dJ/dz, dJ/dE_0) of the oracle `o` (solver settings as set) for
    `nsteps` backward-Euler steps of size dt from u0; weights: (N,) w_c."""
    import scipy.sparse.linalg as spla
    N = o.N
    states = [np.array(u0, dtype=np.float64)]
    for _ in range(nsteps):
        un = states[-1]
        u, st = o.newton(un.copy(), un.copy(), 1.0, dt)
        if st["status"] != 0:
            raise RuntimeError("oracle Newton did not converge: %s" % st)
        states.append(u)
    J = float(np.dot(weights, states[-1][:N]))
    leaf = o.leaf_mask()
    idx = np.nonzero(np.concatenate([leaf, leaf]))[0]
    g = np.zeros(2 * N)
    g[:N] = weights
    g[np.concatenate([~leaf, ~leaf])] = 0.0
    dz = np.zeros(N)
    for n in reversed(range(nsteps)):
        Ju, Jz = o.jacobian(states[n + 1], 1.0, dt)
        M = Ju[idx][:, idx]
        A = M.T.tocsr()
        rhs = g[idx]
        dg = A.diagonal()
        P = spla.LinearOperator(A.shape, lambda v: v / dg)
        x, info = spla.gmres(A, rhs, M=P, rtol=1e-14, atol=0.0, restart=80, maxiter=200)
        res = np.linalg.norm(A @ x - rhs)
        if info != 0 or res > 1e-12 * max(np.linalg.norm(rhs), 1e-300):
            raise RuntimeError("adjoint solve: info %d, residual %.3e" % (info, res))
        lam = np.zeros(2 * N)
        lam[idx] = x
        dz -= Jz[idx].T @ lam[idx]
        g = lam
    return J, dz, g[:N].copy()
