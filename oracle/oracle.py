"""ctypes front end of the plain FP64 CPU oracle (``nrd_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never loads it.

Every method restates a step of arXiv 1302.6303 (see the header of
``nrd_oracle.cpp`` for the section/equation map and the readings R1-R15).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrd_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_NEUMANN, BC_ROBIN = 0, 1
LIM_WILSON, LIM_PAPER_LITERAL = 0, 1
JV_FD, JV_ANALYTIC = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_ubyte)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no FP contraction), with
    OpenMP for its independent cell loops when the compiler has it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                _SRC]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build_oracle())
    vp = ctypes.c_void_p
    sig = {
        "orc_create": (vp, [ctypes.c_int, _ip, _ip, _ip, _dp, ctypes.c_double, ctypes.c_int]),
        "orc_destroy": (None, [vp]),
        "orc_set_threads": (ctypes.c_int, [ctypes.c_int]),
        "orc_ncells": (ctypes.c_long, [vp]),
        "orc_set_material": (None, [vp, _fp]),
        "orc_set_solver": (None, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int]),
        "orc_leaf_mask": (None, [vp, _up]),
        "orc_set_smoother": (None, [vp, ctypes.c_int, ctypes.c_double]),
        "orc_residual": (None, [vp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
        "orc_residual_scale": (None, [vp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
        "orc_jv_analytic": (None, [vp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
        "orc_jv_scale": (None, [vp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
        "orc_fd_eps": (ctypes.c_double, [vp, _dp, _dp]),
        "orc_vjp": (None, [vp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]),
        "orc_set_material_f64": (None, [vp, _dp]),
        "orc_time_derivative": (None, [vp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
        "orc_predict": (None, [vp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
        "orc_lte": (ctypes.c_double, [vp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double]),
        "orc_jv_fd": (ctypes.c_double, [vp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                        _dp, _dp]),
        "orc_dot": (ctypes.c_double, [vp, _dp, _dp]),
        "orc_ghosts": (ctypes.c_long, [vp, _dp, _dp, _dp, _fp]),
        "orc_pc_setup": (None, [vp, _dp, ctypes.c_double, ctypes.c_double]),
        "orc_pc_apply": (None, [vp, _dp, _dp]),
        "orc_comp_apply": (None, [vp, ctypes.c_int, _dp, _dp]),
        "orc_level_apply": (None, [vp, ctypes.c_int, ctypes.c_int, _dp, _dp]),
        "orc_jacobian": (ctypes.c_long, [vp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                         _ip, _ip, _dp]),
        "orc_fac": (None, [vp, ctypes.c_int, _dp, _dp]),
        "orc_gmg": (None, [vp, ctypes.c_int, _dp, _dp]),
        "orc_average_down": (None, [vp, _dp]),
        "orc_newton": (ctypes.c_int, [vp, _dp, _dp, ctypes.c_double, ctypes.c_double, _ip, _ip,
                                      _dp, _dp]),
        "orc_tag": (None, [vp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _up]),
        "orc_tag_values": (None, [vp, _dp, _dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def set_threads(n):
    """Host threads for the oracle's independent cell loops (results are
    bit-identical for any count); returns the count in use (1 when the oracle
    was built without OpenMP)."""
    return _load().orc_set_threads(int(n))


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Oracle:
    """One hierarchy + material field, with the method's operators on it."""

    def __init__(self, hier, z=None, kcond=0.01, limiter=LIM_WILSON):
        lib = _load()
        self.hier = hier
        nb = np.ascontiguousarray(hier.nboxes, dtype=np.int32)
        bx = np.ascontiguousarray(hier.boxes_flat(), dtype=np.int32)
        bt = np.ascontiguousarray(hier.bc_type, dtype=np.int32)
        br = np.ascontiguousarray(hier.bc_R, dtype=np.float64)
        h = lib.orc_create(hier.nlevels, nb.ctypes.data_as(_ip), bx.ctypes.data_as(_ip),
                           bt.ctypes.data_as(_ip), br.ctypes.data_as(_dp), kcond, limiter)
        if not h:
            raise ValueError("oracle rejected the hierarchy")
        self._h = h
        self.N = lib.orc_ncells(h)
        assert self.N == hier.ncells
        if z is not None:
            self.set_material(z)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    def set_material(self, z):
        z = np.ascontiguousarray(z, dtype=np.float32)
        assert z.size == self.N
        _lib.orc_set_material(self._h, z.ctypes.data_as(_fp))

    def set_solver(self, restart=30, max_krylov=300, jv_mode=JV_FD, nu1=2, nu2=2, nmg=4,
                   coarse_sweeps=None, rtol=1e-8, atol=0.0, max_newton=20):
        if coarse_sweeps is None:
            coarse_sweeps = nu1 + nu2
        _lib.orc_set_solver(self._h, restart, max_krylov, jv_mode, nu1, nu2, nmg, coarse_sweeps,
                            rtol, atol, max_newton)

    def set_smoother(self, kind=0, omega=6.0 / 7.0):
        """V-cycle smoother: 0 red-black Gauss-Seidel, 1 damped point Jacobi,
        2 block (x-line) Gauss-Seidel on the box levels (reading R26)."""
        _lib.orc_set_smoother(self._h, kind, omega)

    def leaf_mask(self):
        m = np.zeros(self.N, dtype=np.uint8)
        _lib.orc_leaf_mask(self._h, m.ctypes.data_as(_up))
        return m.astype(bool)

    def residual(self, u, b, a0, dt):
        F = np.empty(2 * self.N)
        _lib.orc_residual(self._h, _d(u), _d(b), a0, dt, _d(F))
        return F

    def residual_scale(self, u, b, a0, dt):
        S = np.empty(2 * self.N)
        _lib.orc_residual_scale(self._h, _d(u), _d(b), a0, dt, _d(S))
        return S

    def jv_analytic(self, u, v, a0, dt):
        J = np.empty(2 * self.N)
        _lib.orc_jv_analytic(self._h, _d(u), _d(v), a0, dt, _d(J))
        return J

    def jv_scale(self, u, v, a0, dt):
        S = np.empty(2 * self.N)
        _lib.orc_jv_scale(self._h, _d(u), _d(v), a0, dt, _d(S))
        return S

    def set_material_f64(self, z):
        z = np.ascontiguousarray(z, dtype=np.float64)
        _lib.orc_set_material_f64(self._h, _d(z))

    def vjp(self, u, w, a0, dt, with_dz=True):
        """(dF/du)^T w, (dF/dz)^T w and sum_i |w_i J_ij| (brute force, small N)."""
        JTw = np.empty(2 * self.N)
        Jab = np.empty(2 * self.N)
        dz = np.empty(self.N) if with_dz else None
        _lib.orc_vjp(self._h, _d(u), _d(np.ascontiguousarray(w)), a0, dt, _d(JTw), _d(dz), _d(Jab))
        return JTw, dz, Jab

    def time_derivative(self, u_np1, u_n, u_nm1, dt, dt_prev=0.0):
        out = np.empty(2 * self.N)
        _lib.orc_time_derivative(self._h, _d(u_np1), _d(u_n), _d(u_nm1), dt, dt_prev, _d(out))
        return out

    def predict(self, u_n, u_nm1, udot_n, dt, dt_prev):
        out = np.empty(2 * self.N)
        _lib.orc_predict(self._h, _d(u_n), _d(u_nm1), _d(udot_n), dt, dt_prev, _d(out))
        return out

    def lte(self, u_np1, u_p, alpha, eta_E=1e-5, eta_T=1e-3):
        return _lib.orc_lte(self._h, _d(u_np1), _d(u_p), alpha, eta_E, eta_T)

    def fd_eps(self, u, v):
        return _lib.orc_fd_eps(self._h, _d(u), _d(v))

    def jv_fd(self, u, v, b, a0, dt, F0=None):
        J = np.empty(2 * self.N)
        eps = _lib.orc_jv_fd(self._h, _d(u), _d(v), _d(b), a0, dt, _d(F0), _d(J))
        return J, eps

    def dot(self, x, y):
        return _lib.orc_dot(self._h, _d(x), _d(y))

    def ghosts(self, u):
        G = self.hier.nghosts
        gE, gT = np.empty(G), np.empty(G)
        gz = np.empty(G, dtype=np.float32)
        n = _lib.orc_ghosts(self._h, _d(u), _d(gE), _d(gT), gz.ctypes.data_as(_fp))
        assert n == G
        return gE, gT, gz

    def pc_setup(self, u, a0, dt):
        _lib.orc_pc_setup(self._h, _d(u), a0, dt)

    def pc_apply(self, w):
        y = np.empty(2 * self.N)
        _lib.orc_pc_apply(self._h, _d(w), _d(y))
        return y

    def comp_apply(self, fld, x):
        y = np.empty(self.N)
        _lib.orc_comp_apply(self._h, fld, _d(np.ascontiguousarray(x)), _d(y))
        return y

    def jacobian(self, u, a0, dt):
        """Sparse dF/du (2N x 2N) and dF/dz (2N x N) at u, every entry the
        residual reaches (scipy CSR)."""
        import scipy.sparse as sp
        u = np.ascontiguousarray(u, dtype=np.float64)
        n2 = 2 * self.N
        cap = 64 * n2
        while True:
            rows = np.empty(cap, dtype=np.int32)
            cols = np.empty(cap, dtype=np.int32)
            vals = np.empty(cap)
            nnz = _lib.orc_jacobian(self._h, _d(u), a0, dt, cap, rows.ctypes.data_as(_ip),
                                    cols.ctypes.data_as(_ip), _d(vals))
            if nnz >= 0:
                break
            cap = -nnz
        rows, cols, vals = rows[:nnz], cols[:nnz], vals[:nnz]
        zc = cols >= n2
        Ju = sp.csr_matrix((vals[~zc], (rows[~zc], cols[~zc])), shape=(n2, n2))
        Jz = sp.csr_matrix((vals[zc], (rows[zc], cols[zc] - n2)), shape=(n2, self.N))
        return Ju, Jz

    def level_apply(self, fld, lev, x):
        """The FAC level operator of level `lev` (homogeneous coarse-fine
        ghosts) on a vector dense over that level's index space."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.size == int(np.prod(self.hier.level_n(lev)))
        y = np.empty_like(x)
        _lib.orc_level_apply(self._h, fld, lev, _d(x), _d(y))
        return y

    def fac(self, fld, f):
        u = np.empty(self.N)
        _lib.orc_fac(self._h, fld, _d(np.ascontiguousarray(f)), _d(u))
        return u

    def gmg(self, fld, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        e = np.empty_like(f)
        _lib.orc_gmg(self._h, fld, _d(f), _d(e))
        return e

    def average_down(self, x):
        x = np.array(x, dtype=np.float64)
        _lib.orc_average_down(self._h, _d(x))
        return x

    def newton(self, u0, b, a0, dt):
        u = np.array(u0, dtype=np.float64)
        ni, ki = ctypes.c_int(0), ctypes.c_int(0)
        f0, f1 = ctypes.c_double(0), ctypes.c_double(0)
        rc = _lib.orc_newton(self._h, _d(u), _d(b), a0, dt, ctypes.byref(ni), ctypes.byref(ki),
                             ctypes.byref(f0), ctypes.byref(f1))
        return u, dict(status=rc, newton_its=ni.value, krylov_its=ki.value, fnorm0=f0.value,
                       fnorm=f1.value)

    def tag_values(self, u):
        """Per cell (rows) the indicators tau^c / (0.1 max|E|),
        tau^g / (0.1 max|E|) and h|grad E|/E that the tags compare."""
        ind = np.empty(3 * self.N)
        _lib.orc_tag_values(self._h, _d(np.ascontiguousarray(u)), _d(ind))
        return ind.reshape(self.N, 3)

    def tag(self, u, thr_c=np.inf, thr_g=np.inf, thr_r=np.inf):
        t = np.zeros(self.N, dtype=np.uint8)
        _lib.orc_tag(self._h, _d(u), thr_c, thr_g, thr_r, t.ctypes.data_as(_up))
        return t
