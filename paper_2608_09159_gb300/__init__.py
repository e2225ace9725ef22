"""Python binding of the GB300 conic-QP PDHG library (include/cqp.h).

Argument marshalling only: every step of the method runs in the CUDA library
libcqp_gb300.so.  The library must have been built (``build()``); importing
the functions below without it raises instead of falling back to anything.

Functions keep the C names: cqp_default_options, cqp_setup, cqp_solve,
cqp_kkt, cqp_free, cqp_spmv, cqp_project, cqp_status_string, cqp_last_error.
`Solver` wraps them for instance dicts (see the `instances` package layout):
host numpy arrays, or torch CUDA tensors for device-resident inputs.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

__all__ = ["build", "lib", "cqp_default_options", "cqp_setup", "cqp_solve", "cqp_kkt", "cqp_free", "cqp_spmv",
           "cqp_project", "cqp_status_string", "cqp_last_error", "cqp_kernel_launches", "Solver", "CQPError",
           "STATUS"]

CQP_OK, CQP_ITER_LIMIT, CQP_TIME_LIMIT = 0, 1, 2
STATUS = {0: "converged", 1: "iteration limit", 2: "time limit", -1: "invalid input", -2: "CUDA error",
          -3: "out of device memory", -4: "non-finite value", -5: "device wait expired", -6: "unsupported"}


class CQPError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("cqp error %d (%s)%s" % (code, STATUS.get(code, "?"), (": " + msg) if msg else ""))
        self.code = code


class CSR(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("val", C.c_void_p)]


class QOp(C.Structure):
    _fields_ = [("diag", C.c_void_p), ("P", CSR), ("rank", C.c_int64), ("R", C.c_void_p), ("D", C.c_void_p)]


class Cones(C.Structure):
    _fields_ = [("nblocks", C.c_int64), ("type", C.c_void_p), ("start", C.c_void_p), ("dim", C.c_void_p),
                ("alpha", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("update", C.c_int32), ("rho", C.c_double),
                ("ruiz_iters", C.c_int32), ("pc_alpha", C.c_double), ("bound_obj", C.c_int32),
                ("rescaled_cones", C.c_int32),
                ("eps0_in", C.c_double), ("gamma_in", C.c_double), ("eps_min_in", C.c_double),
                ("jacobi", C.c_int32), ("max_inner", C.c_int32), ("force_inner", C.c_int32),
                ("beta_s", C.c_double), ("beta_n", C.c_double), ("beta_a", C.c_double),
                ("beta_I", C.c_double), ("K_P", C.c_double), ("K_I", C.c_double), ("K_D", C.c_double),
                ("pid", C.c_int32), ("avg_epoch", C.c_int32),
                ("tol", C.c_double), ("max_iter", C.c_int64), ("check_every", C.c_int32),
                ("time_limit_s", C.c_double),
                ("power_iters", C.c_int32), ("power_tol", C.c_double), ("step_factor", C.c_double),
                ("input_on_device", C.c_int32), ("team", C.c_int32), ("threads", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("tpr_a", C.c_int32), ("tpr_at", C.c_int32), ("tpr_p", C.c_int32),
                ("launch_iters", C.c_int32), ("profile", C.c_int32), ("warm_roots", C.c_int32), ("col_blocks", C.c_int32),
                ("matrix_bf16", C.c_int32),
                ("stream", C.c_void_p)]


class KKTReport(C.Structure):
    _fields_ = [("eps_p", C.c_double), ("eps_d", C.c_double), ("eps_g", C.c_double), ("rel_kkt", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("norm_res_p", C.c_double), ("norm_res_d", C.c_double)]


class Bounds(C.Structure):
    _fields_ = [("row_lo", C.c_void_p), ("row_hi", C.c_void_p), ("x_lo", C.c_void_p), ("x_hi", C.c_void_p)]


class Batch(C.Structure):
    _fields_ = [("count", C.c_int64), ("x_off", C.c_void_p), ("row_off", C.c_void_p)]


class InstanceResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int64), ("restarts", C.c_int64), ("inner_total", C.c_int64),
                ("kkt", KKTReport)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int64), ("restarts", C.c_int64), ("inner_total", C.c_int64),
                ("kernel_launches", C.c_int64), ("kkt", KKTReport), ("eta", C.c_double), ("norm_A", C.c_double),
                ("omega", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("phase_ms", C.c_double * 16), ("kernel_ms", C.c_double), ("setup_launches", C.c_int64)]


_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in-tree)."""
    return _build.build(force=force, verbose=verbose)


def lib():
    """Load libcqp_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libcqp_gb300.so is not built; run paper_2608_09159_gb300.build()")
        L = C.CDLL(_build.LIB)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.cqp_default_options.argtypes = [vp]
        L.cqp_setup.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.cqp_solve.argtypes = [vp, vp, vp, vp, vp, i32, vp]
        L.cqp_kkt.argtypes = [vp, vp, vp, i32, vp]
        L.cqp_free.argtypes = [vp]
        L.cqp_free.restype = None
        L.cqp_status_string.argtypes = [C.c_int]
        L.cqp_status_string.restype = C.c_char_p
        L.cqp_last_error.argtypes = []
        L.cqp_last_error.restype = C.c_char_p
        L.cqp_spmv.argtypes = [i32, i64, i64, vp, vp, vp, vp, vp, i32, vp]
        L.cqp_project.argtypes = [i32, i64, vp, vp, vp, vp, vp]
        L.cqp_kernel_launches.argtypes = []
        L.cqp_kernel_launches.restype = C.c_longlong
        L.cqp_kkt_static.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.cqp_setup_batch.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.cqp_setup_general.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.cqp_solve_batch.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp]
        f32 = C.c_float
        L.cqp_ws_features.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp]
        L.cqp_gemm_bf16.argtypes = [i32, i32, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, i32, i32, vp]
        L.cqp_ws_head_forward.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.cqp_ws_loss.argtypes = [i64, vp, vp, vp, vp, vp, f32, f32, vp, vp, vp, vp]
        L.cqp_ws_head_backward.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.cqp_relu_backward_bf16.argtypes = [i64, i64, vp, vp, vp, vp]
        L.cqp_adam_step.argtypes = [i64, vp, vp, vp, vp, f32, f32, f32, f32, i64, vp, vp]
        L.cqp_ws_start.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, f32, i32, vp, vp, vp]
        L.cqp_gemm_check.argtypes = [vp]
        L.cqp_transpose_bf16.argtypes = [i64, i64, vp, vp, vp]
        L.cqp_umma_smem_desc.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, i32]
        L.cqp_umma_smem_desc.restype = C.c_uint64
        L.cqp_umma_instr_desc_bf16.argtypes = [i32, i32]
        L.cqp_umma_instr_desc_bf16.restype = C.c_uint32
        L.cqp_spmv_merge.argtypes = [i32, i64, i64, vp, vp, vp, vp, vp, vp]
        L.cqp_sell_build.argtypes = [i32, i64, i64, vp, vp, vp, vp, vp]
        L.cqp_sell_stored.argtypes = [vp, vp]
        L.cqp_spmv_sell.argtypes = [vp, vp, vp, vp]
        L.cqp_sell_free.argtypes = [vp]
        L.cqp_sell_free.restype = None
        L.cqp_gemm_tc_launches.argtypes = []
        L.cqp_gemm_tc_launches.restype = C.c_longlong
        for f in ("cqp_default_options", "cqp_setup", "cqp_solve", "cqp_kkt", "cqp_spmv", "cqp_project",
                  "cqp_kkt_static", "cqp_setup_batch", "cqp_solve_batch", "cqp_setup_general", "cqp_ws_features",
                  "cqp_gemm_bf16",
                  "cqp_ws_head_forward", "cqp_ws_loss", "cqp_ws_head_backward", "cqp_relu_backward_bf16",
                  "cqp_adam_step", "cqp_ws_start", "cqp_gemm_check", "cqp_transpose_bf16", "cqp_spmv_merge",
                  "cqp_sell_build", "cqp_sell_stored", "cqp_spmv_sell"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def cqp_status_string(code: int) -> str:
    return lib().cqp_status_string(code).decode()


def cqp_last_error() -> str:
    return lib().cqp_last_error().decode()


def cqp_kernel_launches() -> int:
    return int(lib().cqp_kernel_launches())


def _check(rc, allow_positive=True):
    if rc < 0 or (rc > 0 and not allow_positive):
        raise CQPError(rc, cqp_last_error())
    return rc


def cqp_default_options(**kw) -> Options:
    o = Options()
    _check(lib().cqp_default_options(C.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def cqp_setup(A: CSR, Q, c, b, K: Cones, opt: Options):
    h = C.c_void_p()
    _check(lib().cqp_setup(C.byref(A), None if Q is None else C.byref(Q), c, b, C.byref(K), C.byref(opt), C.byref(h)))
    return h


def cqp_solve(h, x0, y0, x_out, y_out, on_device: int, res: Result) -> int:
    return _check(lib().cqp_solve(h, x0, y0, x_out, y_out, on_device, C.byref(res)))


def cqp_kkt(h, x, y, on_device: int, rep: KKTReport) -> int:
    return _check(lib().cqp_kkt(h, x, y, on_device, C.byref(rep)))


def cqp_setup_general(A: CSR, Q, c, bounds: Bounds, K: Cones, opt: Options):
    h = C.c_void_p()
    _check(lib().cqp_setup_general(C.byref(A), None if Q is None else C.byref(Q), c, C.byref(bounds), C.byref(K),
                                   C.byref(opt), C.byref(h)))
    return h


def cqp_setup_batch(A: CSR, Q, c, b, K: Cones, B: Batch, opt: Options):
    h = C.c_void_p()
    _check(lib().cqp_setup_batch(C.byref(A), None if Q is None else C.byref(Q), c, b, C.byref(K), C.byref(B),
                                 C.byref(opt), C.byref(h)))
    return h


def cqp_solve_batch(h, x0, y0, x_out, y_out, on_device: int, per_instance, res: Result) -> int:
    return _check(lib().cqp_solve_batch(h, x0, y0, x_out, y_out, on_device, per_instance, C.byref(res)))


def cqp_ws_features(count, x_off, n_assets, asset_off, row_off, rank, c, q, R, ldr, b, X, stream=None) -> int:
    return _check(lib().cqp_ws_features(count, x_off, n_assets, asset_off, row_off, rank, c, q, R, ldr, b, X, stream))


def cqp_gemm_bf16(trans_a, trans_b, M, N, K, A, lda, B, ldb, Cm, ldc, bias, epilogue, split_k=1, stream=None) -> int:
    return _check(lib().cqp_gemm_bf16(trans_a, trans_b, M, N, K, A, lda, B, ldb, Cm, ldc, bias, epilogue, split_k,
                                      stream))


def cqp_ws_head_forward(count, asset_off, H2, w3, b3, Wd, bd, score, x0, pooled, ydual, stream=None) -> int:
    return _check(lib().cqp_ws_head_forward(count, asset_off, H2, w3, b3, Wd, bd, score, x0, pooled, ydual, stream))


def cqp_ws_loss(count, asset_off, x0, xstar, ydual, ystar, lam, scale, dscore, dydual, loss, stream=None) -> int:
    return _check(lib().cqp_ws_loss(count, asset_off, x0, xstar, ydual, ystar, lam, scale, dscore, dydual, loss,
                                    stream))


def cqp_ws_head_backward(count, asset_off, H2, w3, Wd, dscore, dydual, pooled, dZ2, gw3, gb3, gWd, gbd,
                         stream=None) -> int:
    return _check(lib().cqp_ws_head_backward(count, asset_off, H2, w3, Wd, dscore, dydual, pooled, dZ2, gw3, gb3,
                                             gWd, gbd, stream))


def cqp_relu_backward_bf16(rows, cols, H, dH, gbias, stream=None) -> int:
    return _check(lib().cqp_relu_backward_bf16(rows, cols, H, dH, gbias, stream))


def cqp_adam_step(n, w, g, m, v, lr, beta1, beta2, eps, step, w_bf16, stream=None) -> int:
    return _check(lib().cqp_adam_step(n, w, g, m, v, lr, beta1, beta2, eps, step, w_bf16, stream))


def cqp_ws_start(count, x_off, row_off, n_assets, asset_off, rank, q, R, ldr, b, xw, ydual, yb_scale, dual_mode, x0,
                 y0, stream=None) -> int:
    return _check(lib().cqp_ws_start(count, x_off, row_off, n_assets, asset_off, rank, q, R, ldr, b, xw, ydual,
                                     yb_scale, dual_mode, x0, y0, stream))


def cqp_gemm_check(stream=None) -> int:
    """Raises if a bounded wait inside a tensor-memory GEMM expired since the last check."""
    return _check(lib().cqp_gemm_check(stream))


def cqp_transpose_bf16(rows, cols, src, dst, stream=None) -> int:
    return _check(lib().cqp_transpose_bf16(rows, cols, src, dst, stream))


def cqp_spmv_merge(precision, nrows, ncols, rowptr, colind, val, x, y, stream=None) -> int:
    return _check(lib().cqp_spmv_merge(precision, nrows, ncols, rowptr, colind, val, x, y, stream))


class Sell:
    """Sliced-ELL copy of a device CSR matrix (cqp_sell_build / cqp_spmv_sell / cqp_sell_free)."""

    def __init__(self, precision, nrows, ncols, rowptr, colind, val, stream=None):
        self.h = C.c_void_p()
        _check(lib().cqp_sell_build(precision, nrows, ncols, rowptr, colind, val, stream, C.byref(self.h)))
        n = C.c_int64()
        _check(lib().cqp_sell_stored(self.h, C.byref(n)))
        self.stored = n.value

    def spmv(self, x, y, stream=None):
        return _check(lib().cqp_spmv_sell(self.h, x, y, stream))

    def close(self):
        if self.h:
            lib().cqp_sell_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cqp_free(h) -> None:
    lib().cqp_free(h)


def cqp_spmv(precision, nrows, ncols, rowptr, colind, val, x, y, threads_per_row=0, stream=None) -> int:
    return _check(lib().cqp_spmv(precision, nrows, ncols, rowptr, colind, val, x, y, threads_per_row, stream))


def cqp_project(precision, n, K_device: Cones, r, m, out, stream=None) -> int:
    return _check(lib().cqp_project(precision, n, C.byref(K_device), r, m, out, stream))


def cqp_kkt_static(A_device: CSR, Q_device, c, b, K_device: Cones, x, y, rep: KKTReport, stream=None) -> int:
    """Allocation-free KKT report from device arrays (for callers that must not cudaMalloc)."""
    return _check(lib().cqp_kkt_static(C.byref(A_device), None if Q_device is None else C.byref(Q_device), c, b,
                                       C.byref(K_device), x, y, C.byref(rep), stream))


# ---------------------------------------------------------------------------
# convenience wrapper over instance dicts
# ---------------------------------------------------------------------------

def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Solver:
    """Owns a cqp_handle built from an instance dict.

    Host numpy arrays are passed as host pointers.  With ``device=True`` the
    arrays are first copied to torch CUDA tensors and passed as device pointers
    (``input_on_device = 1``), i.e. the inputs are resident in HBM.
    """

    def __init__(self, inst, device: bool = False, **opts):
        self._keep = []
        self.inst = inst
        self.n, self.m = int(inst["n"]), int(inst["m"])
        conv = {
            "a_rowptr": np.int64, "a_colind": np.int32, "a_val": np.float64, "c": np.float64, "b": np.float64,
            "q_diag": np.float64, "q_R": np.float64, "q_D": np.float64, "p_rowptr": np.int64, "p_colind": np.int32,
            "p_val": np.float64, "blk_type": np.int32, "blk_start": np.int64, "blk_dim": np.int64,
            "blk_alpha": np.float64, "row_lo": np.float64, "row_hi": np.float64, "x_lo": np.float64,
            "x_hi": np.float64}
        arrs = {}
        for k, dt in conv.items():
            v = inst.get(k)
            if v is None:
                arrs[k] = None
                continue
            if hasattr(v, "data_ptr"):
                arrs[k] = v
            else:
                arrs[k] = np.ascontiguousarray(v, dtype=dt)
        if device:
            import torch
            for k, v in list(arrs.items()):
                if v is not None and not hasattr(v, "data_ptr"):
                    arrs[k] = torch.from_numpy(v).cuda()
        if device or any(getattr(v, "is_cuda", False) for v in arrs.values() if v is not None):
            opts["input_on_device"] = 1
        self._keep.append(arrs)
        p = _ptr
        self.A = CSR(self.m, self.n, int(inst["a_rowptr"][-1]), p(arrs["a_rowptr"]), p(arrs["a_colind"]),
                     p(arrs["a_val"]))
        R = arrs["q_R"]
        rank = 0 if R is None else int(R.shape[0])
        Pm = CSR(self.n, self.n, 0 if arrs["p_rowptr"] is None else int(inst["p_rowptr"][-1]),
                 p(arrs["p_rowptr"]), p(arrs["p_colind"]), p(arrs["p_val"]))
        self.Q = QOp(p(arrs["q_diag"]), Pm, rank, p(R), p(arrs["q_D"]))
        self.K = Cones(int(len(inst["blk_type"])), p(arrs["blk_type"]), p(arrs["blk_start"]), p(arrs["blk_dim"]),
                       p(arrs["blk_alpha"]))
        self.opt = cqp_default_options(**opts)
        self.h = self._setup(arrs)

    def _setup(self, arrs):
        if any(arrs.get(k) is not None for k in ("row_lo", "row_hi", "x_lo", "x_hi")):
            self.G = Bounds(_ptr(arrs.get("row_lo")), _ptr(arrs.get("row_hi")), _ptr(arrs.get("x_lo")),
                            _ptr(arrs.get("x_hi")))
            return cqp_setup_general(self.A, self.Q, _ptr(arrs["c"]), self.G, self.K, self.opt)
        return cqp_setup(self.A, self.Q, _ptr(arrs["c"]), _ptr(arrs["b"]), self.K, self.opt)

    def solve(self, x0=None, y0=None, out_device=False):
        """Returns (x, y, result dict).  With out_device the outputs are torch CUDA tensors."""
        res = Result()
        if out_device:
            import torch
            x = torch.empty(self.n, dtype=torch.float64, device="cuda")
            y = torch.empty(max(self.m, 1), dtype=torch.float64, device="cuda")
            x0p = None if x0 is None else x0.data_ptr()
            y0p = None if y0 is None else y0.data_ptr()
            rc = cqp_solve(self.h, x0p, y0p, x.data_ptr(), y.data_ptr(), 1, res)
            y = y[:self.m]
        else:
            x = np.zeros(self.n)
            y = np.zeros(self.m)
            x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
            y0 = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
            rc = cqp_solve(self.h, _ptr(x0), _ptr(y0), _ptr(x), _ptr(y), 0, res)
        return x, y, result_dict(res, rc)

    def kkt(self, x, y):
        rep = KKTReport()
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        cqp_kkt(self.h, _ptr(x), _ptr(y), 0, rep)
        return {f: getattr(rep, f) for f, _ in KKTReport._fields_}

    def close(self):
        if getattr(self, "h", None):
            cqp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver(Solver):
    """Owns a batch handle (cqp_setup_batch) built from a block-diagonal batch
    instance dict (keys of an instance plus batch_count, x_off, row_off)."""

    def _setup(self, arrs):
        inst = self.inst
        self.count = int(inst["batch_count"])
        self._xo = np.ascontiguousarray(inst["x_off"], dtype=np.int64)
        self._ro = np.ascontiguousarray(inst["row_off"], dtype=np.int64)
        self.B = Batch(self.count, self._xo.ctypes.data, self._ro.ctypes.data)
        return cqp_setup_batch(self.A, self.Q, _ptr(arrs["c"]), _ptr(arrs["b"]), self.K, self.B, self.opt)

    def solve(self, x0=None, y0=None, out_device=False):
        """Returns (x, y, per-instance list of dicts, summary result dict)."""
        res = Result()
        per = (InstanceResult * self.count)()
        if out_device:
            import torch
            x = torch.empty(self.n, dtype=torch.float64, device="cuda")
            y = torch.empty(max(self.m, 1), dtype=torch.float64, device="cuda")
            rc = cqp_solve_batch(self.h, None if x0 is None else x0.data_ptr(), None if y0 is None else y0.data_ptr(),
                                 x.data_ptr(), y.data_ptr(), 1, per, res)
            y = y[:self.m]
        else:
            x = np.zeros(self.n)
            y = np.zeros(self.m)
            x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
            y0 = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
            rc = cqp_solve_batch(self.h, _ptr(x0), _ptr(y0), _ptr(x), _ptr(y), 0, per, res)
        plist = [{"rc": r.status, "iters": r.iters, "restarts": r.restarts, "inner_total": r.inner_total,
                  "kkt": {f: getattr(r.kkt, f) for f, _ in KKTReport._fields_}} for r in per]
        return x, y, plist, result_dict(res, rc)


def result_dict(res: Result, rc: int):
    d = {f: getattr(res, f) for f, _ in Result._fields_ if f not in ("kkt", "phase_ms")}
    d["phase_ms"] = list(res.phase_ms)
    d["kkt"] = {f: getattr(res.kkt, f) for f, _ in KKTReport._fields_}
    d["rc"] = rc
    return d
