"""Thin Python binding of the nrd C ABI (include/nrd.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libnrd.so``.  Tensors are torch CUDA tensors (device memory and the
current stream come from torch); nothing here falls back to a CPU path, and
loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libnrd.so")

OK, EINVAL, ENOMEM, ENONCONV, ENEG, ENAN, ECUDA, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
BC_NEUMANN, BC_ROBIN = 0, 1
LIM_WILSON, LIM_PAPER_LITERAL = 0, 1
JV_FD, JV_ANALYTIC, JV_FROZEN = 0, 1, 2
PC_F64, PC_F32 = 0, 1
SMOOTH_RBGS, SMOOTH_JACOBI, SMOOTH_LINE = 0, 1, 2
DT_EPS, DT_PC47 = 0, 1

EXPORTED = [
    "nrd_params_default", "nrd_create", "nrd_destroy", "nrd_last_error", "nrd_set_params",
    "nrd_set_hierarchy", "nrd_layout", "nrd_set_material", "nrd_ghost_fill", "nrd_residual",
    "nrd_jv", "nrd_linearise", "nrd_vjp", "nrd_adjoint_solve", "nrd_fd_eps", "nrd_dot", "nrd_precond_setup", "nrd_precond_apply", "nrd_newton",
    "nrd_step", "nrd_step_begin", "nrd_step_end", "nrd_tag", "nrd_regrid_boxes", "nrd_transfer", "nrd_time_derivative", "nrd_predict", "nrd_lte", "nrd_dt_control",
    "nrd_autotune", "nrd_autotune_sweeps", "nrd_wdot_noalloc", "nrd_measure_peaks",
    "nrd_measure_fp64_ops",
    "nrd_check_fastmath", "nrd_check_narrow",
    "nrd_timing_enable",
    "nrd_timing_read",
]
TK_RESIDUAL, TK_JV, TK_JV_FD, TK_PC_APPLY, TK_PC_SETUP, TK_ORTHO, TK_GHOST, TK_TRANSFER = range(8)
TK_NAMES = ["residual", "jv", "jv_fd", "pc_apply", "pc_setup", "ortho", "ghost", "transfer",
            "linearise"]


class Params(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_double), ("limiter", ctypes.c_int), ("u_min", ctypes.c_double),
        ("restart", ctypes.c_int), ("max_krylov", ctypes.c_int), ("jv_mode", ctypes.c_int),
        ("pc_precision", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
        ("nmg", ctypes.c_int), ("coarse_sweeps", ctypes.c_int), ("rtol", ctypes.c_double),
        ("atol", ctypes.c_double), ("max_newton", ctypes.c_int), ("eta_max", ctypes.c_double),
        ("ew_gamma", ctypes.c_double), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
        ("tile_z", ctypes.c_int), ("graph", ctypes.c_int), ("smoother", ctypes.c_int),
        ("omega", ctypes.c_double), ("eta0", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("newton_its", ctypes.c_int), ("krylov_its", ctypes.c_int),
        ("pc_setups", ctypes.c_int), ("fnorm0", ctypes.c_double), ("fnorm", ctypes.c_double),
        ("min_lambda", ctypes.c_double), ("kernels", ctypes.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NrdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("nrd error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path: str = _LIBPATH):
    """Load libnrd.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libnrd.so not built: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, dp, fp = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    c_int, c_dbl = ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "nrd_params_default": (c_int, [P(Params)]),
        "nrd_create": (c_int, [P(Params), P(vp)]),
        "nrd_destroy": (c_int, [vp]),
        "nrd_last_error": (ctypes.c_char_p, [vp]),
        "nrd_set_params": (c_int, [vp, P(Params)]),
        "nrd_set_hierarchy": (c_int, [vp, c_int, P(c_int), P(c_int), P(c_int), P(c_dbl)]),
        "nrd_layout": (c_int, [vp, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)]),
        "nrd_set_material": (c_int, [vp, fp, vp]),
        "nrd_ghost_fill": (c_int, [vp, dp, dp, dp, fp, vp]),
        "nrd_residual": (c_int, [vp, dp, dp, c_dbl, c_dbl, dp, vp]),
        "nrd_jv": (c_int, [vp, dp, dp, dp, dp, c_dbl, c_dbl, c_int, dp, vp]),
        "nrd_linearise": (c_int, [vp, dp, dp, c_dbl, c_dbl, dp, vp]),
        "nrd_vjp": (c_int, [vp, dp, c_dbl, c_dbl, dp, dp, vp]),
        "nrd_adjoint_solve": (c_int, [vp, dp, c_dbl, c_dbl, c_dbl, dp, P(Stats), vp]),
        "nrd_fd_eps": (c_int, [vp, dp, dp, P(c_dbl), vp]),
        "nrd_dot": (c_int, [vp, dp, dp, P(c_dbl), vp]),
        "nrd_precond_setup": (c_int, [vp, dp, c_dbl, c_dbl, vp]),
        "nrd_precond_apply": (c_int, [vp, dp, dp, vp]),
        "nrd_newton": (c_int, [vp, dp, dp, c_dbl, c_dbl, P(Stats), vp]),
        "nrd_step": (c_int, [vp, dp, dp, dp, c_dbl, c_dbl, P(Stats), vp]),
        "nrd_step_begin": (c_int, [vp, dp, dp, dp, c_dbl, c_dbl, vp]),
        "nrd_step_end": (c_int, [vp, P(Stats)]),
        "nrd_tag": (c_int, [vp, dp, c_dbl, c_dbl, c_dbl, vp, vp]),
        "nrd_regrid_boxes": (c_int, [vp, vp, c_int, c_int, c_dbl, c_int, c_int, c_int, c_int,
                                     P(c_int), P(c_int), P(c_int), P(c_int)]),
        "nrd_transfer": (c_int, [vp, vp, dp, dp, c_int, vp]),
        "nrd_autotune": (c_int, [vp, dp, dp, c_dbl, c_dbl, P(c_int), P(c_dbl), vp]),
        "nrd_autotune_sweeps": (c_int, [vp, dp, dp, c_dbl, c_dbl, P(c_int), P(c_dbl), vp]),
        "nrd_time_derivative": (c_int, [vp, dp, dp, dp, c_dbl, c_dbl, dp, vp]),
        "nrd_predict": (c_int, [vp, dp, dp, dp, c_dbl, c_dbl, dp, vp]),
        "nrd_lte": (c_int, [vp, dp, dp, c_dbl, c_dbl, c_dbl, P(c_dbl), vp]),
        "nrd_dt_control": (c_int, [c_int, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, P(c_dbl)]),
        "nrd_wdot_noalloc": (c_int, [dp, dp, fp, ctypes.c_int64, dp, vp]),
        "nrd_measure_peaks": (c_int, [P(c_dbl), P(c_dbl), P(c_dbl), vp]),
        "nrd_measure_fp64_ops": (c_int, [P(c_dbl), vp]),
        "nrd_check_fastmath": (c_int, [dp, ctypes.c_int64, dp, vp]),
        "nrd_check_narrow": (c_int, [dp, ctypes.c_int64, fp, vp]),
        "nrd_timing_enable": (c_int, [vp, c_int]),
        "nrd_timing_read": (c_int, [vp, c_int, P(c_dbl), P(ctypes.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_params(**kw) -> Params:
    lib = load()
    p = Params()
    lib.nrd_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t, dtype):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous() and t.dtype == dtype):
        raise ValueError("expected a contiguous CUDA tensor of dtype %s" % dtype)
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def measure_peaks():
    """FP64 / FP32 FMA TFLOP/s and copy GB/s of the current device."""
    lib = load()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib.nrd_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream())
    if rc != OK:
        raise NrdError(rc, "nrd_measure_peaks failed")
    return {"fp64_tflops": a.value, "fp32_tflops": b.value, "copy_gbs": c.value}


def measure_fp64_ops():
    """FP64 FMA, division and square-root rates (operations per second) of
    the current device."""
    lib = load()
    r = (ctypes.c_double * 3)()
    rc = lib.nrd_measure_fp64_ops(r, _stream())
    if rc != OK:
        raise NrdError(rc, "nrd_measure_fp64_ops failed")
    return {"fma_per_s": r[0], "div_per_s": r[1], "sqrt_per_s": r[2]}


def check_fastmath(x):
    """[rcp(x), 1/x, rsqrt(x), 1/sqrt(x)] as evaluated by the stencil's
    refined reciprocals and by CUDA's rounded operations (nrd_check_fastmath)."""
    out = torch.empty(4, x.numel(), dtype=torch.float64, device=x.device)
    rc = load().nrd_check_fastmath(_ptr(x, torch.float64), x.numel(), _ptr(out, torch.float64),
                                   _stream())
    if rc != OK:
        raise NrdError(rc, "nrd_check_fastmath failed")
    return out


def check_narrow(x):
    """[narrow(x), (float) x]: the stencil's integer-instruction FP64 -> FP32
    round-to-nearest-even narrowing and CUDA's conversion (nrd_check_narrow)."""
    out = torch.empty(2, x.numel(), dtype=torch.float32, device=x.device)
    rc = load().nrd_check_narrow(_ptr(x, torch.float64), x.numel(), _ptr(out, torch.float32),
                                 _stream())
    if rc != OK:
        raise NrdError(rc, "nrd_check_narrow failed")
    return out


def dt_control(kind, eps_t, err_n, err_nm1, dt_n, dt_nm1):
    """EPS (Eq. odets) or PC.4.7 (Eq. pc47) step-size controller."""
    out = ctypes.c_double()
    rc = load().nrd_dt_control(kind, eps_t, err_n, err_nm1, dt_n, dt_nm1, ctypes.byref(out))
    if rc != OK:
        raise NrdError(rc, "nrd_dt_control: bad arguments")
    return out.value


def wdot_noalloc(x, y, w, out=None):
    """Allocation-free weighted dot (nrd_wdot_noalloc): out[0] =
    sum_i w_i (x_i y_i + x_{n+i} y_{n+i}); returns the 1-element device tensor."""
    lib = load()
    n = w.numel()
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=x.device)
    rc = lib.nrd_wdot_noalloc(_ptr(x, torch.float64), _ptr(y, torch.float64), _ptr(w, torch.float32),
                              n, _ptr(out, torch.float64), _stream())
    if rc != OK:
        raise NrdError(rc, "nrd_wdot_noalloc failed")
    return out


class Context:
    """One nrd context: a hierarchy, a material field and solver state."""

    def __init__(self, params: Params | None = None, **kw):
        self.lib = load()
        self.params = params if params is not None else default_params(**kw)
        h = ctypes.c_void_p()
        rc = self.lib.nrd_create(ctypes.byref(self.params), ctypes.byref(h))
        if rc != OK:
            raise NrdError(rc, "nrd_create failed (bad parameters?)")
        self._h = h
        self.N = self.G = self.nleaf = self.nlevels = 0

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.nrd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            msg = self.lib.nrd_last_error(self._h)
            raise NrdError(rc, msg.decode() if msg else "")
        return rc

    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        self._check(self.lib.nrd_set_params(self._h, ctypes.byref(self.params)))

    def set_hierarchy(self, nboxes, boxes, bc_type, bc_R):
        nb = (ctypes.c_int * len(nboxes))(*nboxes)
        bx = (ctypes.c_int * len(boxes))(*boxes)
        bt = (ctypes.c_int * 6)(*bc_type)
        br = (ctypes.c_double * 6)(*bc_R)
        self._check(self.lib.nrd_set_hierarchy(self._h, len(nboxes), nb, bx, bt, br))
        n, g, lf = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.nrd_layout(self._h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(lf)))
        self.N, self.G, self.nleaf = n.value, g.value, lf.value
        self.nlevels = len(nboxes)

    def set_hierarchy_from(self, hier):
        self.set_hierarchy(hier.nboxes, hier.boxes_flat(), hier.bc_type, hier.bc_R)

    def set_material(self, z):
        self._check(self.lib.nrd_set_material(self._h, _ptr(z, torch.float32), _stream()))

    def ghost_fill(self, u):
        gE = torch.empty(self.G, dtype=torch.float64, device=u.device)
        gT = torch.empty_like(gE)
        gz = torch.empty(self.G, dtype=torch.float32, device=u.device)
        self._check(self.lib.nrd_ghost_fill(self._h, _ptr(u, torch.float64), _ptr(gE, torch.float64),
                                            _ptr(gT, torch.float64), _ptr(gz, torch.float32),
                                            _stream()))
        return gE, gT, gz

    def residual(self, u, b, a0, dt, out=None):
        out = torch.empty_like(u) if out is None else out
        self._check(self.lib.nrd_residual(self._h, _ptr(u, torch.float64), _ptr(b, torch.float64),
                                          a0, dt, _ptr(out, torch.float64), _stream()))
        return out

    def jv(self, u, v, a0, dt, mode=JV_ANALYTIC, b=None, F0=None, out=None):
        out = torch.empty_like(u) if out is None else out
        self._check(self.lib.nrd_jv(self._h, _ptr(u, torch.float64), _ptr(v, torch.float64),
                                    _ptr(b, torch.float64), _ptr(F0, torch.float64), a0, dt, mode,
                                    _ptr(out, torch.float64), _stream()))
        return out

    def linearise(self, u, b, a0, dt, out=None):
        out = torch.empty_like(u) if out is None else out
        self._check(self.lib.nrd_linearise(self._h, _ptr(u, torch.float64), _ptr(b, torch.float64),
                                           a0, dt, _ptr(out, torch.float64), _stream()))
        return out

    def vjp(self, w, a0, dt, out=None, dz=None, want_dz=True):
        """(dF/du)^T w and (dF/dz)^T w at the last linearisation."""
        out = torch.empty_like(w) if out is None else out
        if want_dz and dz is None:
            dz = torch.empty(self.N, dtype=torch.float64, device=w.device)
        self._check(self.lib.nrd_vjp(self._h, _ptr(w, torch.float64), a0, dt,
                                     _ptr(out, torch.float64), _ptr(dz, torch.float64), _stream()))
        return out, dz

    def adjoint_solve(self, g, a0, dt, rtol=1e-10, out=None, check=True):
        """Solve J^T lam = g at the last linearisation."""
        out = torch.empty_like(g) if out is None else out
        st = Stats()
        rc = self.lib.nrd_adjoint_solve(self._h, _ptr(g, torch.float64), a0, dt, rtol,
                                        _ptr(out, torch.float64), ctypes.byref(st), _stream())
        if check and rc != OK:
            self._check(rc)
        return out, st.as_dict()

    def fd_eps(self, u, v):
        e = ctypes.c_double()
        self._check(self.lib.nrd_fd_eps(self._h, _ptr(u, torch.float64), _ptr(v, torch.float64),
                                        ctypes.byref(e), _stream()))
        return e.value

    def dot(self, x, y):
        d = ctypes.c_double()
        self._check(self.lib.nrd_dot(self._h, _ptr(x, torch.float64), _ptr(y, torch.float64),
                                     ctypes.byref(d), _stream()))
        return d.value

    def precond_setup(self, u, a0, dt):
        self._check(self.lib.nrd_precond_setup(self._h, _ptr(u, torch.float64), a0, dt, _stream()))

    def precond_apply(self, w, out=None):
        out = torch.empty_like(w) if out is None else out
        self._check(self.lib.nrd_precond_apply(self._h, _ptr(w, torch.float64),
                                               _ptr(out, torch.float64), _stream()))
        return out

    def newton(self, u, b, a0, dt, check=True):
        st = Stats()
        rc = self.lib.nrd_newton(self._h, _ptr(u, torch.float64), _ptr(b, torch.float64), a0, dt,
                                 ctypes.byref(st), _stream())
        if check and rc not in (OK,):
            self._check(rc)
        return st.as_dict()

    def step(self, u, u_n, u_nm1, dt, dt_prev=0.0, check=True):
        st = Stats()
        rc = self.lib.nrd_step(self._h, _ptr(u, torch.float64), _ptr(u_n, torch.float64),
                               _ptr(u_nm1, torch.float64), dt, dt_prev, ctypes.byref(st), _stream())
        if check and rc != OK:
            self._check(rc)
        return st.as_dict()

    def step_begin(self, u, u_n, u_nm1, dt, dt_prev=0.0):
        """Enqueue one implicit step on the current stream without waiting
        (nrd_step_begin); finish it with step_end()."""
        self._check(self.lib.nrd_step_begin(self._h, _ptr(u, torch.float64),
                                            _ptr(u_n, torch.float64), _ptr(u_nm1, torch.float64),
                                            dt, dt_prev, _stream()))

    def step_end(self, check=True):
        """Wait for the step begun by step_begin(); its stats (nrd_step_end)."""
        st = Stats()
        rc = self.lib.nrd_step_end(self._h, ctypes.byref(st))
        if check and rc != OK:
            self._check(rc)
        return st.as_dict()

    def autotune(self, u, b, a0, dt):
        """Pick the fastest stencil tile shape for this hierarchy at state u."""
        t = (ctypes.c_int * 3)()
        ms = ctypes.c_double()
        self._check(self.lib.nrd_autotune(self._h, _ptr(u, torch.float64), _ptr(b, torch.float64),
                                          a0, dt, t, ctypes.byref(ms), _stream()))
        self.params.tile_x, self.params.tile_y, self.params.tile_z = t[0], t[1], t[2]
        return (t[0], t[1], t[2]), ms.value

    def autotune_sweeps(self, u_n, u_nm1, dt, dt_prev=0.0):
        """Pick the fastest smoother and sweep schedule for one implicit step;
        returns ((nu1, nu2, coarse_sweeps, smoother), ms)."""
        nu = (ctypes.c_int * 4)()
        ms = ctypes.c_double()
        self._check(self.lib.nrd_autotune_sweeps(self._h, _ptr(u_n, torch.float64),
                                                 _ptr(u_nm1, torch.float64), dt, dt_prev, nu,
                                                 ctypes.byref(ms), _stream()))
        self.params.nu1, self.params.nu2, self.params.coarse_sweeps = nu[0], nu[1], nu[2]
        self.params.smoother = nu[3]
        return (nu[0], nu[1], nu[2], nu[3]), ms.value

    def time_derivative(self, u_np1, u_n, u_nm1, dt, dt_prev=0.0, out=None):
        out = torch.empty_like(u_n) if out is None else out
        self._check(self.lib.nrd_time_derivative(self._h, _ptr(u_np1, torch.float64),
                                                 _ptr(u_n, torch.float64),
                                                 _ptr(u_nm1, torch.float64), dt, dt_prev,
                                                 _ptr(out, torch.float64), _stream()))
        return out

    def predict(self, u_n, u_nm1, udot_n, dt, dt_prev, out=None):
        out = torch.empty_like(u_n) if out is None else out
        self._check(self.lib.nrd_predict(self._h, _ptr(u_n, torch.float64),
                                         _ptr(u_nm1, torch.float64), _ptr(udot_n, torch.float64),
                                         dt, dt_prev, _ptr(out, torch.float64), _stream()))
        return out

    def lte(self, u_np1, u_p, alpha, eta_E=1e-5, eta_T=1e-3):
        e = ctypes.c_double()
        self._check(self.lib.nrd_lte(self._h, _ptr(u_np1, torch.float64), _ptr(u_p, torch.float64),
                                     alpha, eta_E, eta_T, ctypes.byref(e), _stream()))
        return e.value

    def timing_enable(self, on=True):
        self._check(self.lib.nrd_timing_enable(self._h, 1 if on else 0))

    def timing_read(self):
        out = {}
        for k, name in enumerate(TK_NAMES):
            ms, n = ctypes.c_double(), ctypes.c_int64()
            self._check(self.lib.nrd_timing_read(self._h, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def tag(self, u, thr_c=float("inf"), thr_g=float("inf"), thr_r=float("inf")):
        t = torch.empty(self.N, dtype=torch.uint8, device=u.device)
        self._check(self.lib.nrd_tag(self._h, _ptr(u, torch.float64), thr_c, thr_g, thr_r,
                                     _ptr(t, torch.uint8), _stream()))
        return t

    def regrid_boxes(self, tags, tag_bits=1, buffer=1, efficiency=0.7, min_side=4, max_side=32,
                     max_levels=None, max_boxes=4096):
        """Berger-Rigoutsos boxes of a new hierarchy from device tags
        (nrd_regrid_boxes); returns levels[l] = [(lo, hi), ...]."""
        if max_levels is None:
            max_levels = self.nlevels
        nl, tot = ctypes.c_int(), ctypes.c_int()
        nb = (ctypes.c_int * max_levels)()
        bx = (ctypes.c_int * (6 * max_boxes))()
        self._check(self.lib.nrd_regrid_boxes(self._h, _ptr(tags, torch.uint8), tag_bits, buffer,
                                              efficiency, min_side, max_side, max_levels,
                                              max_boxes, ctypes.byref(nl), nb, bx,
                                              ctypes.byref(tot)))
        out, q = [], 0
        for l in range(nl.value):
            lev = []
            for _ in range(nb[l]):
                lev.append((tuple(bx[6 * q:6 * q + 3]), tuple(bx[6 * q + 3:6 * q + 6])))
                q += 1
            out.append(lev)
        return out

    def transfer_to(self, dst: "Context", u):
        """Conservative limited-linear transfer (nrd_transfer) of one state
        vector or a stack of them (shape (nvec, 2N)) to dst's hierarchy."""
        stacked = u.dim() == 2
        uu = u.contiguous() if stacked else u.reshape(1, -1).contiguous()
        nvec = uu.shape[0]
        out = torch.empty(nvec, 2 * dst.N, dtype=torch.float64, device=u.device)
        rc = self.lib.nrd_transfer(self._h, dst._h, _ptr(uu, torch.float64),
                                   _ptr(out, torch.float64), nvec, _stream())
        dst._check(rc)
        return out if stacked else out[0]
