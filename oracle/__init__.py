"""Python access to the plain FP64 C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2608_09159_gb300``) never does.  The oracle shares no code with the
CUDA library; both sides only consume the same seeded instances.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")

FREE, NONNEG, SOC, RSOC, EXP, POW = 0, 1, 2, 3, 4, 5
# slices with the middle coordinate fixed (eq. fisher-conic): {(r, f, t): f e^(r/f) <= t} and
# {(x, f, z): x^a f^(1-a) >= |z|, x >= 0}, f = blk_fix (1 by default)
EXP1, POW1 = 7, 8


def build(force: bool = False, omp: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so, or with -fopenmp into
    liboracle_omp.so (the same source; used to time the CPU baseline on all host cores)."""
    out = _OUT_OMP if omp else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + ".%d.tmp" % os.getpid()
        flags = ["-fopenmp"] if omp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", *flags, "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class Problem(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64),
                ("a_rowptr", C.c_void_p), ("a_colind", C.c_void_p), ("a_val", C.c_void_p),
                ("q_diag", C.c_void_p),
                ("p_rowptr", C.c_void_p), ("p_colind", C.c_void_p), ("p_val", C.c_void_p),
                ("q_rank", C.c_int64), ("q_R", C.c_void_p), ("q_D", C.c_void_p),
                ("c", C.c_void_p), ("b", C.c_void_p),
                ("nblocks", C.c_int64),
                ("blk_type", C.c_void_p), ("blk_start", C.c_void_p), ("blk_dim", C.c_void_p),
                ("blk_alpha", C.c_void_p),
                ("row_lo", C.c_void_p), ("row_hi", C.c_void_p), ("x_lo", C.c_void_p), ("x_hi", C.c_void_p),
                ("blk_fix", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("ruiz_iters", C.c_int), ("pc_alpha", C.c_double), ("bound_obj", C.c_int),
                ("eps0_in", C.c_double), ("gamma_in", C.c_double), ("eps_min_in", C.c_double),
                ("jacobi", C.c_int), ("rho", C.c_double),
                ("beta_s", C.c_double), ("beta_n", C.c_double), ("beta_a", C.c_double),
                ("beta_I", C.c_double), ("K_P", C.c_double), ("K_I", C.c_double), ("K_D", C.c_double),
                ("check_every", C.c_int), ("max_iter", C.c_int64), ("max_inner", C.c_int),
                ("tol", C.c_double), ("update", C.c_int), ("avg_epoch", C.c_int),
                ("power_iters", C.c_int), ("power_tol", C.c_double), ("step_factor", C.c_double),
                ("force_inner", C.c_int), ("pid", C.c_int), ("hist_cap", C.c_int), ("rescaled_cones", C.c_int)]


class KKT(C.Structure):
    _fields_ = [("eps_p", C.c_double), ("eps_d", C.c_double), ("eps_g", C.c_double),
                ("rel_kkt", C.c_double), ("pobj", C.c_double), ("dobj", C.c_double),
                ("norm_res_p", C.c_double), ("norm_res_d", C.c_double)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int64), ("restarts", C.c_int64),
                ("inner_total", C.c_int64), ("eta", C.c_double), ("norm_A", C.c_double),
                ("omega", C.c_double), ("beta_b", C.c_double), ("beta_c", C.c_double),
                ("kkt", KKT), ("hist_len", C.c_int),
                ("hist_iter", C.c_void_p), ("hist_kkt", C.c_void_p), ("hist_gap", C.c_void_p),
                ("hist_E", C.c_void_p), ("hist_restart", C.c_void_p)]


_libs = {}
_use_omp = False


def use_openmp(flag: bool = True, threads: int = 0) -> int:
    """Route the wrappers below to the OpenMP build (flag) with `threads` threads (0: the
    runtime's default); returns the thread count a parallel loop will use."""
    global _use_omp
    _use_omp = bool(flag)
    lb = lib()
    if flag and threads > 0:
        lb.orc_set_threads(int(threads))
    return int(lb.orc_max_threads())


def lib():
    omp = _use_omp
    if omp not in _libs:
        _libs[omp] = _load(build(omp=omp))
    return _libs[omp]


def _load(path):
    _lib = C.CDLL(path)
    _lib.orc_proj_block.restype = C.c_int
    _lib.orc_in_cone.restype = C.c_int
    _lib.orc_in_dual_cone.restype = C.c_int
    _lib.orc_norm_est.restype = C.c_double
    _lib.orc_pdhg_operator.restype = C.c_int
    _lib.orc_prox.restype = C.c_int
    _lib.orc_solve.restype = C.c_int
    for fn in ("orc_in_cone", "orc_in_dual_cone"):
        getattr(_lib, fn).argtypes = [C.c_int, C.c_int64, C.c_double, C.c_void_p, C.c_double]
    _lib.orc_proj_block.argtypes = [C.c_int, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
    _lib.orc_proj_block_scaled.restype = C.c_int
    _lib.orc_proj_block_scaled.argtypes = [C.c_int, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p]
    _lib.orc_power_start.argtypes = [C.c_int64, C.c_void_p]
    _lib.orc_tridiag_max_eig.restype = C.c_double
    _lib.orc_tridiag_max_eig.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    _lib.orc_norm_est.argtypes = [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                  C.c_double, C.c_void_p]
    _lib.orc_pdhg_operator.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                       C.c_double, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    _lib.orc_prox.argtypes = [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                              C.c_int, C.c_int, C.c_void_p]
    vp, i64 = C.c_void_p, C.c_int64
    _lib.orc_default_options.argtypes = [vp]
    _lib.orc_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
    _lib.orc_spmv_t.argtypes = [i64, i64, vp, vp, vp, vp, vp]
    _lib.orc_q_apply.argtypes = [vp, vp, vp]
    _lib.orc_proj_product.argtypes = [vp, vp, vp, vp]
    _lib.orc_kkt.argtypes = [vp, vp, vp, vp]
    _lib.orc_rescale.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    _lib.orc_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    _lib.orc_proj_slice.restype = C.c_int
    _lib.orc_proj_slice.argtypes = [C.c_int, C.c_double, C.c_double, vp, vp, vp]
    _lib.orc_restart_rule.restype = C.c_int
    _lib.orc_restart_rule.argtypes = [C.c_double, C.c_double, C.c_double, i64, i64, vp]
    _lib.orc_pid_update.restype = C.c_double
    _lib.orc_pid_update.argtypes = [C.c_double, C.c_double, C.c_double, vp, vp]
    _lib.orc_inner_tol.restype = C.c_double
    _lib.orc_inner_tol.argtypes = [C.c_double, C.c_double, C.c_double, vp]
    _lib.orc_set_threads.argtypes = [C.c_int]
    _lib.orc_max_threads.restype = C.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Prob:
    """Keeps the numpy arrays of an instance alive while a Problem struct points at them."""

    def __init__(self, inst):
        self.keep = []

        def arr(key, dt):
            v = inst.get(key)
            if v is None:
                return None
            v = np.ascontiguousarray(v, dtype=dt)
            self.keep.append(v)
            return v

        a_rowptr = arr("a_rowptr", np.int64)
        R = arr("q_R", np.float64)
        self.s = Problem(
            m=int(inst["m"]), n=int(inst["n"]),
            a_rowptr=_p(a_rowptr), a_colind=_p(arr("a_colind", np.int64)), a_val=_p(arr("a_val", np.float64)),
            q_diag=_p(arr("q_diag", np.float64)),
            p_rowptr=_p(arr("p_rowptr", np.int64)), p_colind=_p(arr("p_colind", np.int64)),
            p_val=_p(arr("p_val", np.float64)),
            q_rank=0 if R is None else int(R.shape[0]), q_R=_p(R), q_D=_p(arr("q_D", np.float64)),
            c=_p(arr("c", np.float64)), b=_p(arr("b", np.float64)),
            nblocks=int(len(inst["blk_type"])),
            blk_type=_p(arr("blk_type", np.int32)), blk_start=_p(arr("blk_start", np.int64)),
            blk_dim=_p(arr("blk_dim", np.int64)), blk_alpha=_p(arr("blk_alpha", np.float64)),
            row_lo=_p(arr("row_lo", np.float64)), row_hi=_p(arr("row_hi", np.float64)),
            x_lo=_p(arr("x_lo", np.float64)), x_hi=_p(arr("x_hi", np.float64)),
            blk_fix=_p(arr("blk_fix", np.float64)))

    @property
    def ptr(self):
        return C.byref(self.s)


def default_options(**kw) -> Options:
    o = Options()
    lib().orc_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------

def spmv(rowptr, colind, val, x):
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colind = np.ascontiguousarray(colind, np.int64)
    val, x = _f64(val), _f64(x)
    y = np.zeros(rowptr.size - 1)
    lib().orc_spmv(C.c_int64(y.size), _p(rowptr), _p(colind), _p(val), _p(x), _p(y))
    return y


def spmv_t(rowptr, colind, val, y, n):
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colind = np.ascontiguousarray(colind, np.int64)
    val, y = _f64(val), _f64(y)
    out = np.zeros(n)
    lib().orc_spmv_t(C.c_int64(rowptr.size - 1), C.c_int64(n), _p(rowptr), _p(colind), _p(val), _p(y), _p(out))
    return out


def q_apply(inst, x):
    P = _Prob(inst)
    x = _f64(x)
    out = np.zeros(int(inst["n"]))
    lib().orc_q_apply(P.ptr, _p(x), _p(out))
    return out


def proj_block(ctype, r, alpha=0.0, m=None):
    r = _f64(r)
    mm = None if m is None else _f64(m)
    out = np.zeros_like(r)
    rc = lib().orc_proj_block(int(ctype), r.size, float(alpha), _p(r), _p(mm), _p(out))
    if rc != 0:
        raise ValueError("invalid cone block")
    return out


def proj_block_scaled(ctype, sc, r, alpha=0.0, m=None):
    """Projection onto the rescaled cone diag(sc) K in the metric m (eq. scaling-induced-metric)."""
    r, sc = _f64(r), _f64(sc)
    mm = None if m is None else _f64(m)
    out = np.zeros_like(r)
    rc = lib().orc_proj_block_scaled(int(ctype), r.size, float(alpha), _p(sc), _p(r), _p(mm), _p(out))
    if rc != 0:
        raise ValueError("invalid cone block")
    return out


def proj_slice(ctype, r, alpha=0.0, f=1.0, m=None):
    """Projection onto the slice EXP1 / POW1 with middle coordinate f, metric m (None: Euclidean)."""
    r = _f64(r)
    mm = None if m is None else _f64(m)
    out = np.zeros(3)
    rc = lib().orc_proj_slice(int(ctype), float(alpha), float(f), _p(r), _p(mm), _p(out))
    if rc != 0:
        raise ValueError("invalid slice block")
    return out


def restart_rule(E, E0, Eprev, k, ktot, **opts):
    """The oracle's restart decision (eq. practical-restart-rule)."""
    o = default_options(**opts)
    return bool(lib().orc_restart_rule(float(E), float(E0), float(Eprev), int(k), int(ktot), C.byref(o)))


def pid_update(omega, dx, dy, state, **opts):
    """The oracle's primal-weight update (eqs. pid-error, pid-weight); state = [I, e_prev] is updated."""
    o = default_options(**opts)
    st = np.ascontiguousarray(state, dtype=np.float64)
    w = lib().orc_pid_update(float(omega), float(dx), float(dy), C.byref(o), _p(st))
    state[:] = st
    return w


def inner_tol(eps_prev, mov, tau, **opts):
    """The oracle's adaptive inner tolerance (eq. monotone-primal-inner-tol)."""
    o = default_options(**opts)
    return lib().orc_inner_tol(float(eps_prev), float(mov), float(tau), C.byref(o))


def proj_product(inst, r, m=None):
    P = _Prob(inst)
    r = _f64(r)
    mm = None if m is None else _f64(m)
    out = np.zeros_like(r)
    lib().orc_proj_product(P.ptr, _p(r), _p(mm), _p(out))
    return out


def in_cone(ctype, r, alpha=0.0, tol=0.0):
    r = _f64(r)
    return bool(lib().orc_in_cone(int(ctype), r.size, float(alpha), _p(r), float(tol)))


def in_dual_cone(ctype, r, alpha=0.0, tol=0.0):
    r = _f64(r)
    return bool(lib().orc_in_dual_cone(int(ctype), r.size, float(alpha), _p(r), float(tol)))


def kkt(inst, x, y):
    P = _Prob(inst)
    x, y = _f64(x), _f64(y)
    rep = KKT()
    lib().orc_kkt(P.ptr, _p(x), _p(y), C.byref(rep))
    return {f: getattr(rep, f) for f, _ in KKT._fields_}


def rescale(inst, **opts):
    P = _Prob(inst)
    o = default_options(**opts)
    n, m = int(inst["n"]), int(inst["m"])
    col, row, bc = np.zeros(n), np.zeros(m), np.zeros(2)
    av = np.zeros(int(inst["a_rowptr"][-1]))
    c, b = np.zeros(n), np.zeros(m)
    lib().orc_rescale(P.ptr, C.byref(o), _p(col), _p(row), _p(bc), _p(av), _p(c), _p(b))
    return dict(col=col, row=row, beta_b=bc[0], beta_c=bc[1], a_val=av, c=c, b=b)


def tridiag_max_eig(a, b):
    a, b = _f64(a), _f64(b if len(b) else np.zeros(1))
    return lib().orc_tridiag_max_eig(_p(a), _p(b), a.size)


def power_start(n):
    out = np.zeros(n)
    lib().orc_power_start(n, _p(out))
    return out


def norm_est(rowptr, colind, val, n, iters=200, tol=1e-6):
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colind = np.ascontiguousarray(colind, np.int64)
    val = _f64(val)
    used = C.c_int(0)
    s = lib().orc_norm_est(rowptr.size - 1, n, _p(rowptr), _p(colind), _p(val), iters, tol, C.byref(used))
    return s, used.value


def pdhg_operator(inst, tau, sigma, x, y, eps_in=1e-12, max_inner=100000, jacobi=1, force_inner=0):
    P = _Prob(inst)
    x, y = _f64(x), _f64(y)
    xo, yo = np.zeros_like(x), np.zeros_like(y)
    it = lib().orc_pdhg_operator(P.ptr, tau, sigma, _p(x), _p(y), eps_in, max_inner, jacobi, force_inner,
                                 _p(xo), _p(yo))
    return xo, yo, it


def prox(inst, tau, v, u0=None, eps_in=1e-12, max_inner=100000, jacobi=1, force_inner=0):
    P = _Prob(inst)
    v = _f64(v)
    u0 = v.copy() if u0 is None else _f64(u0)
    out = np.zeros_like(v)
    it = lib().orc_prox(P.ptr, tau, _p(v), _p(u0), eps_in, max_inner, jacobi, force_inner, _p(out))
    return out, it


def solve(inst, x0=None, y0=None, hist_cap=0, **opts):
    P = _Prob(inst)
    o = default_options(hist_cap=hist_cap, **opts)
    n, m = int(inst["n"]), int(inst["m"])
    x, y = np.zeros(n), np.zeros(m)
    x0 = None if x0 is None else _f64(x0)
    y0 = None if y0 is None else _f64(y0)
    info = Info()
    hist = {}
    if hist_cap:
        hist = dict(iter=np.zeros(hist_cap, np.int64), kkt=np.zeros(hist_cap), gap=np.zeros(hist_cap),
                    E=np.zeros(hist_cap), restart=np.zeros(hist_cap, np.int32))
        info.hist_iter, info.hist_kkt, info.hist_gap = _p(hist["iter"]), _p(hist["kkt"]), _p(hist["gap"])
        info.hist_E, info.hist_restart = _p(hist["E"]), _p(hist["restart"])
    lib().orc_solve(P.ptr, C.byref(o), _p(x0), _p(y0), _p(x), _p(y), C.byref(info))
    out = {f: getattr(info, f) for f, _ in Info._fields_ if not f.startswith("hist") and f != "kkt"}
    out["kkt"] = {f: getattr(info.kkt, f) for f, _ in KKT._fields_}
    if hist_cap:
        L = info.hist_len
        out["hist"] = {k: v[:L].copy() for k, v in hist.items()}
    return x, y, out
