"""GPU test of cqp_kkt_static, the KKT entry point that allocates no device memory.

Callers that may not call cudaMalloc (for instance code inside a framework
that already owns the device memory pool, or code that must keep a fixed
device footprint) cannot build a handle, so cqp_kkt is closed to them.
cqp_kkt_static gives them the same report from their own device arrays, using
a static scratch array of the library.  This file checks, through the C ABI,
that its report matches cqp_kkt on a handle within the tolerance of the other
KKT test, on two calls in a row (the scratch keeps the previous call's contents,
so the second call shows the clearing works), on problems of different sizes
back to back, and that sizes beyond the static limit are refused before any
kernel runs.  The file is named so that pytest collects it last.
"""

import numpy as np
import pytest

import instances as I

pytestmark = pytest.mark.gpu

FIELDS = ("eps_p", "eps_d", "eps_g", "rel_kkt", "pobj", "dobj", "norm_res_p", "norm_res_d")


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_09159_gb300 as g
    g.build()
    g.lib()
    return g


def _device_problem(g, inst):
    """Device copies of the instance arrays and the C structs that point at them."""
    import torch

    def dev(key, dt):
        v = inst.get(key)
        return None if v is None else torch.from_numpy(np.ascontiguousarray(v, dtype=dt)).cuda()

    t = {k: dev(k, dt) for k, dt in (
        ("a_rowptr", np.int64), ("a_colind", np.int32), ("a_val", np.float64), ("c", np.float64),
        ("b", np.float64), ("q_diag", np.float64), ("q_R", np.float64), ("q_D", np.float64),
        ("p_rowptr", np.int64), ("p_colind", np.int32), ("p_val", np.float64), ("blk_type", np.int32),
        ("blk_start", np.int64), ("blk_dim", np.int64), ("blk_alpha", np.float64))}
    p = lambda a: None if a is None else a.data_ptr()
    n, m = int(inst["n"]), int(inst["m"])
    A = g.CSR(m, n, int(inst["a_rowptr"][-1]), p(t["a_rowptr"]), p(t["a_colind"]), p(t["a_val"]))
    pnnz = 0 if inst.get("p_rowptr") is None else int(inst["p_rowptr"][-1])
    P = g.CSR(n, n, pnnz, p(t["p_rowptr"]), p(t["p_colind"]), p(t["p_val"]))
    rank = 0 if inst.get("q_R") is None else int(inst["q_R"].shape[0])
    Q = g.QOp(p(t["q_diag"]), P, rank, p(t["q_R"]), p(t["q_D"]))
    K = g.Cones(len(inst["blk_type"]), p(t["blk_type"]), p(t["blk_start"]), p(t["blk_dim"]), p(t["blk_alpha"]))
    return A, Q, K, t


def _static_report(g, prob, x, y):
    import torch
    A, Q, K, t = prob
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    rep = g.KKTReport()
    g.cqp_kkt_static(A, Q, t["c"].data_ptr(), t["b"].data_ptr(), K, xd.data_ptr(), yd.data_ptr(), rep)
    return {f: getattr(rep, f) for f in FIELDS}


def _point(inst, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=inst["n"]), rng.normal(size=inst["m"])


def _close(got, ref):
    for f in FIELDS:
        if not np.isfinite(ref[f]):        # e.g. a dual objective of -inf (slice support term)
            assert got[f] == ref[f], (f, got[f], ref[f])
            continue
        assert abs(got[f] - ref[f]) <= 1e-10 * (1.0 + abs(ref[f])), (f, got[f], ref[f])


@pytest.mark.parametrize("k", [1, 2, 3])
def test_two_calls_match_handle_kkt(gpu, orc, k):
    inst = I.small_config(k)      # k = 3: exponential and power slice blocks
    x, y = _point(inst, 40 + k)
    s = gpu.Solver(inst, precision=1)
    ref = s.kkt(x, y)
    s.close()
    prob = _device_problem(gpu, inst)
    first = _static_report(gpu, prob, x, y)
    second = _static_report(gpu, prob, x, y)
    _close(first, ref)
    _close(second, ref)
    _close(first, orc.kkt(inst, x, y))          # and the FP64 oracle's report of the same point


def test_malformed_row_pointers_are_reported(gpu):
    # a row pointer past nnz (or a first entry other than 0) is flagged and its row skipped:
    # the call reads only the caller's nnz entries and returns CQP_ERR_INVALID
    import torch
    inst = I.small_config(1)
    x, y = _point(inst, 9)
    for bad_at, value in ((inst["m"], int(inst["a_rowptr"][-1]) + 64), (0, 1)):
        A, Q, K, t = _device_problem(gpu, inst)
        t["a_rowptr"][bad_at] = value
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        rep = gpu.KKTReport()
        with pytest.raises(gpu.CQPError) as e:
            gpu.cqp_kkt_static(A, Q, t["c"].data_ptr(), t["b"].data_ptr(), K, xd.data_ptr(), yd.data_ptr(), rep)
        assert e.value.code == -1 and "malformed" in str(e.value)


def test_back_to_back_sizes_clear_the_scratch(gpu):
    # a larger problem, then a smaller one, then the larger one again: stale
    # entries of the shared scratch beyond the smaller n must not leak in
    big, small = I.small_config(2), I.small_config(3)
    assert big["n"] > small["n"]
    refs = {}
    for name, inst in (("big", big), ("small", small)):
        x, y = _point(inst, 7)
        s = gpu.Solver(inst, precision=1)
        refs[name] = (x, y, s.kkt(x, y))
        s.close()
    pb, ps = _device_problem(gpu, big), _device_problem(gpu, small)
    for name, prob in (("big", pb), ("small", ps), ("big", pb), ("small", ps)):
        x, y, ref = refs[name]
        _close(_static_report(gpu, prob, x, y), ref)


def test_rejects_sizes_beyond_the_static_limit(gpu):
    limit = 524288  # CQP_KKT_STATIC_MAX_N
    n = limit + 1
    dummy = np.zeros(4)
    A = gpu.CSR(0, n, 0, None, None, None)
    K = gpu.Cones(1, None, None, None, None)
    rep = gpu.KKTReport()
    before = gpu.cqp_kernel_launches()
    with pytest.raises(gpu.CQPError) as e:
        gpu.cqp_kkt_static(A, None, dummy.ctypes.data, None, K, dummy.ctypes.data, None, rep)
    assert e.value.code == -1
    assert "exceeds the static scratch limit" in str(e.value)
    assert gpu.cqp_kernel_launches() == before
