"""GPU parity of the BF16 matrix storage (option matrix_bf16: 1 = values of A and A' held in BF16,
2 = also those of the sparse part P of Q; FP32 accumulation, FP32 iterates).

* the BF16-valued SpMV (cqp_spmv, precision 2) against the FP64 oracle on the BF16-rounded
  values, element by element at 1e-5 of the row's |A||x|, for every row width;
* whole solves of scaled-down copies of the sparse QP, SOCP and large-QP workloads: the problem
  solved is the one with A (mode 1) or A and P (mode 2) rounded to BF16 (to FP32, then BF16,
  nearest-even), so the oracle re-measures the returned point on that rounded instance (rel-KKT
  <= 1e-4) and its objective must match the oracle's tight solve of the rounded instance to 1e-4
  relative.  Mode 2 runs on the large QP, whose P (a diagonal plus a weighted matching Laplacian)
  stays positive semidefinite when rounded; the sparse QP's P = M'M + 1e-2 I does not (rounded
  entrywise it has a negative eigenvalue, and the oracle itself diverges on it), so that
  workload runs in mode 1;
* the option's refusals (FP64 iterates, teams other than the whole GPU, unknown modes).
"""
import numpy as np
import pytest

import instances as I
from _parity import REL_KKT, TIGHT_TOL, obj_close

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


def _csr_random(rng, m, n, density, long_rows=0):
    A = (rng.uniform(size=(m, n)) < density) * rng.normal(size=(m, n))
    A[rng.integers(0, m, size=max(1, m // 20))] = 0.0            # empty rows
    for r in rng.integers(0, m, size=long_rows):
        A[r] = rng.normal(size=n)                                   # dense rows
    rows, cols = np.nonzero(A)
    rp = np.zeros(m + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols, A[rows, cols]


@pytest.mark.parametrize("tpr", [-1, 0, 1, 2, 4, 8, 16, 32])
def test_spmv_bf16_matches_oracle_on_rounded_values(gpu, orc, tpr):
    import torch
    rng = np.random.default_rng(500 + tpr)
    m, n = 1537, 1203                                               # ragged tail over many tiles
    rp, ci, v = _csr_random(rng, m, n, 0.01, long_rows=3)
    x = rng.normal(size=n).astype(np.float32)
    vb = I.bf16_bits(v)
    vt = torch.from_numpy(vb.view(np.int16)).cuda()
    xt = torch.from_numpy(x).cuda()
    yt = torch.full((m,), float("nan"), dtype=torch.float32, device="cuda")
    rpt = torch.tensor(rp, dtype=torch.int32, device="cuda")
    cit = torch.tensor(ci, dtype=torch.int32, device="cuda")
    gpu.cqp_spmv(2, m, n, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(), xt.data_ptr(), yt.data_ptr(), tpr)
    vr = I.round_bf16(v)
    xr = x.astype(np.float64)
    ref = orc.spmv(rp, ci, vr, xr)
    scale = orc.spmv(rp, ci, np.abs(vr), np.abs(xr)) + 1e-300
    err = np.abs(yt.double().cpu().numpy() - ref) / scale
    assert err.max() <= 1e-5


@pytest.mark.parametrize("k,mode", [(1, 1), (2, 1), (5, 1), (5, 2)])
def test_bf16_solves_the_rounded_problem(gpu, orc, k, mode):
    # config 1 at full size (n = 1,000): the scaled-down copy has rows with 0-2 entries, and with
    # b = A x0 from the unrounded A its rounded system A x = b, x >= 0 is infeasible (the oracle
    # diverges on it); at full size (3-25 entries per row) the rounded problem stays feasible.
    # Its objective is still 2.4e-4 from the optimum at the first check below 1e-4, so it runs to 1e-5.
    inst = I.sparse_qp_nonneg() if k == 1 else I.small_config(k)
    s = gpu.Solver(inst, precision=0, matrix_bf16=mode, max_iter=400000, tol=1e-5 if k == 1 else 1e-4,
                   time_limit_s=120.0)
    x, y, res = s.solve()
    rep_gpu = s.kkt(x, y)
    s.close()
    assert res["rc"] == 0, res
    rounded = I.with_bf16_matrices(inst, p=mode == 2)
    rep = orc.kkt(rounded, x, y)                 # the rounded instance is the one solved and reported
    assert rep["rel_kkt"] <= REL_KKT, rep
    assert abs(rep["rel_kkt"] - rep_gpu["rel_kkt"]) <= 1e-7 + 1e-3 * rep["rel_kkt"], (rep, rep_gpu)
    xs, ys, info = orc.solve(rounded, max_iter=1000000, tol=TIGHT_TOL)
    assert info["status"] == 0
    assert obj_close(rep["pobj"], info["kkt"]["pobj"]), (rep["pobj"], info["kkt"]["pobj"])
    if k in (1, 2, 5):                            # Q positive definite: x* unique (an extra check)
        assert np.linalg.norm(x - xs) <= 2e-2 * (1 + np.linalg.norm(xs))


@pytest.mark.parametrize("mode", [0, 2])
def test_forced_one_lane_rows_and_column_slices(gpu, orc, mode):
    """The large QP's small copy with the paths its full size takes forced on: one lane per row
    with four rows in flight for A, A' and P (P, with exactly two entries per row, then takes the
    16-byte four-row gradient, head and tail rows the one-row loop) and 5 column slices for A z and
    A'y; FP32 values (mode 0) and BF16 values (mode 2).  Oracle-measured rel-KKT <= 1e-4 on the
    problem solved, and the oracle's tight objective."""
    inst = I.small_config(5)
    s = gpu.Solver(inst, precision=0, matrix_bf16=mode, tpr_a=-1, tpr_at=-1, tpr_p=-1, col_blocks=5, team=1,
                   max_iter=200000, tol=1e-4, time_limit_s=120.0)
    x, y, res = s.solve()
    s.close()
    assert res["rc"] == 0, res
    solved = I.with_bf16_matrices(inst) if mode == 2 else inst
    rep = orc.kkt(solved, x, y)
    assert rep["rel_kkt"] <= REL_KKT, rep
    xs, ys, info = orc.solve(solved, max_iter=1000000, tol=TIGHT_TOL)
    assert obj_close(rep["pobj"], info["kkt"]["pobj"]), (rep["pobj"], info["kkt"]["pobj"])
    assert np.linalg.norm(x - xs) <= 2e-2 * (1 + np.linalg.norm(xs))


def test_bf16_values_already_representable_give_the_same_problem(gpu, orc):
    # an instance whose values are BF16 already: rounding changes nothing, so the KKT report of a
    # point through a BF16 handle equals the oracle's on the instance itself
    inst = I.with_bf16_matrices(I.small_config(5))
    s = gpu.Solver(inst, precision=0, matrix_bf16=2)
    rng = np.random.default_rng(8)
    x, y = rng.normal(size=inst["n"]), rng.normal(size=inst["m"])
    rep = s.kkt(x, y)
    s.close()
    ref = orc.kkt(inst, x, y)
    for key in ("eps_p", "eps_d", "pobj", "dobj"):
        assert abs(rep[key] - ref[key]) <= 1e-5 * (1 + abs(ref[key])), (key, rep[key], ref[key])


def test_bf16_refusals(gpu):
    inst = I.small_config(1)
    with pytest.raises(gpu.CQPError) as e:
        gpu.Solver(inst, precision=1, matrix_bf16=1)
    assert e.value.code == -6
    with pytest.raises(gpu.CQPError) as e:
        gpu.Solver(inst, precision=0, matrix_bf16=1, team=2)
    assert e.value.code == -6
    with pytest.raises(gpu.CQPError) as e:
        gpu.Solver(inst, precision=0, matrix_bf16=3)
    assert e.value.code == -1
