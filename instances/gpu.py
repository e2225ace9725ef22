"""Device-side generation of the large sparse QP (instances.large_qp) on the GPU.

Inputs only: the kernels in gen_gpu.cu draw the same index-addressed Philox values
as the numpy generator, so a small copy generated here equals large_qp(...) of the
same sizes (indices exactly, values to the last bits of log1p / cos).  The arrays
are returned as torch CUDA tensors in an instance dict.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np

from . import CONE_NONNEG, LARGE_NNZ_PER_ROW, blocks_from_list, uniform_at

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen_gpu.cu")
_OUT = os.path.join(_HERE, "_build", "libinstgen.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _OUT + ".%d.tmp" % os.getpid()
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                               "-Xcompiler", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i64, u32 = C.c_void_p, C.c_int64, C.c_uint32
        L.igen_large_qp.argtypes = [u32, i64, i64, i64] + [vp] * 9 + [vp]
        L.igen_large_qp.restype = C.c_int
        _lib = L
    return _lib


def large_qp_device(n=200_000_000, m=50_000_000, seed=1005):
    """instances.large_qp generated in device memory (torch CUDA tensors)."""
    import torch
    assert n % 2 == 0
    k = LARGE_NNZ_PER_ROW
    d = 2 * int(uniform_at(seed, 7, np.zeros(1, dtype=np.uint64))[0] * (n // 2)) + 1
    dev = "cuda"
    t = dict(a_rowptr=torch.empty(m + 1, dtype=torch.int64, device=dev),
             a_colind=torch.empty(m * k, dtype=torch.int32, device=dev),
             a_val=torch.empty(m * k, dtype=torch.float64, device=dev),
             b=torch.empty(m, dtype=torch.float64, device=dev), c=torch.empty(n, dtype=torch.float64, device=dev),
             q_diag=torch.empty(n, dtype=torch.float64, device=dev),
             p_rowptr=torch.empty(n + 1, dtype=torch.int64, device=dev),
             p_colind=torch.empty(2 * n, dtype=torch.int32, device=dev),
             p_val=torch.empty(2 * n, dtype=torch.float64, device=dev))
    rc = _load().igen_large_qp(seed, n, m, d, *(t[x].data_ptr() for x in (
        "a_rowptr", "a_colind", "a_val", "b", "c", "q_diag", "p_rowptr", "p_colind", "p_val")),
        torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise ValueError("igen_large_qp failed (%d)" % rc)
    btype, bstart, bdim, balpha = blocks_from_list([(CONE_NONNEG, n, 0.0)])
    inst = dict(name="large_qp_n%d_m%d" % (n, m), m=m, n=n, blk_type=btype, blk_start=bstart, blk_dim=bdim,
                blk_alpha=balpha, q_R=None, q_D=None)
    inst.update(t)
    return inst
