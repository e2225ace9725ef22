"""GPU parity of the merge-based and sliced-ELL sparse products (cqp_spmv_merge, cqp_sell_*)
against the FP64 oracle, element by element on the same seeded inputs: 1e-12 of the row's
|A||x| in FP64, 1e-5 in FP32 and with BF16 values (compared with the oracle on the rounded
values).  Cases: ragged random rows with empty and dense rows, one row holding every entry (its
sum is split over many threads and blocks and rebuilt from the carries), rows all empty, a
single entry, and the row-length profile of the large QP's A' (Poisson-like, 5 per row).
"""
import numpy as np
import pytest

import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_09159_gb300 as g
    g.build()
    g.lib()
    return g


def _random_csr(rng, m, n, density, long_rows=0):
    A = (rng.uniform(size=(m, n)) < density) * rng.normal(size=(m, n))
    A[rng.integers(0, m, size=max(1, m // 20))] = 0.0
    for r in rng.integers(0, m, size=long_rows):
        A[r] = rng.normal(size=n)
    rows, cols = np.nonzero(A)
    rp = np.zeros(m + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols.astype(np.int64), A[rows, cols]


def _cases():
    rng = np.random.default_rng(77)
    yield "ragged", 1537, 1203, *_random_csr(rng, 1537, 1203, 0.01, long_rows=3)
    n = 60000                                              # one row with every entry
    yield "one_long_row", 3, n, np.array([0, 0, n, n]), np.arange(n), rng.normal(size=n)
    yield "all_empty", 70, 50, np.zeros(71, np.int64), np.zeros(0, np.int64), np.zeros(0)
    yield "single_entry", 5, 4, np.array([0, 0, 0, 1, 1, 1]), np.array([2]), np.array([1.5])
    m, n2 = 40000, 10000                                   # Poisson row lengths, mean 5
    lens = rng.poisson(5.0, size=m)
    rp = np.concatenate([[0], np.cumsum(lens)])
    yield "poisson_rows", m, n2, rp, rng.integers(0, n2, size=rp[-1]), rng.normal(size=rp[-1])


CASES = list(_cases())


def _run(gpu, kind, precision, m, n, rp, ci, v, x):
    import torch
    dt = {0: torch.float32, 1: torch.float64, 2: torch.float32}[precision]
    vd = v if len(v) else np.zeros(1)                      # device arrays of at least one entry
    if precision == 2:
        vt = torch.from_numpy(I.bf16_bits(vd).view(np.int16)).cuda()
        vr = I.round_bf16(v)
    else:
        vt = torch.tensor(vd, dtype=dt, device="cuda")
        vr = vt.double().cpu().numpy()[:len(v)]
    xt = torch.tensor(x, dtype=dt, device="cuda")
    yt = torch.full((m,), float("nan"), dtype=dt, device="cuda")
    rpt = torch.tensor(rp, dtype=torch.int32, device="cuda")
    cit = torch.tensor(ci if len(ci) else np.zeros(1, np.int64), dtype=torch.int32, device="cuda")
    if kind == "merge":
        gpu.cqp_spmv_merge(precision, m, n, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(), xt.data_ptr(),
                           yt.data_ptr())
    else:
        A = gpu.Sell(precision, m, n, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr())
        lens = np.diff(rp)
        want = sum(32 * int(lens[s:s + 32].max()) for s in range(0, m, 32)) if m else 0
        assert A.stored == want
        A.spmv(xt.data_ptr(), yt.data_ptr())
        torch.cuda.synchronize()
        A.close()
    return yt.double().cpu().numpy(), vr, xt.double().cpu().numpy()


@pytest.mark.parametrize("kind", ["merge", "sell"])
@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_variant_matches_oracle(gpu, orc, kind, precision, case):
    name, m, n, rp, ci, v = CASES[case]
    x = np.random.default_rng(case).normal(size=n)
    got, vr, xr = _run(gpu, kind, precision, m, n, rp, ci, v, x)
    ref = orc.spmv(rp, ci, vr, xr)
    scale = orc.spmv(rp, ci, np.abs(vr), np.abs(xr)) + 1e-300
    err = np.abs(got - ref) / scale
    assert np.all(np.isfinite(got)), name
    assert err.max() <= (1e-12 if precision == 1 else 1e-5), (name, err.max())
    empty = np.diff(rp) == 0
    assert np.all(got[empty] == 0.0), name


def test_merge_is_deterministic(gpu):
    name, m, n, rp, ci, v = CASES[1]                       # the row split over many threads
    x = np.random.default_rng(5).normal(size=n)
    a, _, _ = _run(gpu, "merge", 0, m, n, rp, ci, v, x)
    b, _, _ = _run(gpu, "merge", 0, m, n, rp, ci, v, x)
    assert np.array_equal(a, b)
