"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py times.

The oracle cannot run these solves in test time. Instead:
* SOCP mix (n = 200,000, m = 100,000, 2.0M nnz): the FP32 solve's returned point has its
  KKT re-measured by the FP64 oracle. The solver's SpMV over the full A is checked against
  the oracle's FP64 product. Cone projections of the full cone layout (2,000 SOC, 500 RSOC
  blocks) are checked on sampled blocks.
* Fisher market (10,000 buyers x 1,000 goods): the FP32 and FP64 solves reach rel-KKT <= 1e-4
  as re-measured by the oracle, with the objective of the oracle's tol-1e-7 solve (stored by
  tests/golden/make_fisher_objective.py) to 1e-4 relative; exp / pow slice and cone projections
  of the full layouts are checked on sampled blocks.
* Portfolio batch (4,096 instances, 137M nnz, one launch): sampled instances have their KKT
  re-measured by the oracle on the instance alone.
* QCQP front-end workload (n = 202,600): the returned point's KKT is re-measured by the
  oracle.
"""
import numpy as np
import pytest

import _cones as G
import instances as I
from _parity import REL_KKT, obj_close

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


def _device(inst):
    import torch
    keys = ("a_rowptr", "a_colind", "a_val", "c", "b", "q_diag", "q_R", "q_D", "p_rowptr", "p_colind", "p_val",
            "blk_type", "blk_start", "blk_dim", "blk_alpha", "row_lo", "row_hi", "x_lo", "x_hi")
    out = {}
    for k, v in inst.items():
        if k in keys and hasattr(v, "dtype"):
            dt = {"a_colind": np.int32, "p_colind": np.int32, "blk_type": np.int32}.get(k, v.dtype)
            out[k] = torch.from_numpy(np.ascontiguousarray(v, dtype=dt)).cuda()
        else:
            out[k] = v
    return out


@pytest.fixture(scope="module")
def socp():
    return I.socp_mix()


def test_socp_mix_full_solve(gpu, orc, socp):
    s = gpu.Solver(_device(socp), precision=0, tol=1e-4, max_iter=200000, time_limit_s=600.0)
    x, y, res = s.solve(out_device=True)
    s.close()
    assert res["rc"] == 0, res
    rep = orc.kkt(socp, x.double().cpu().numpy(), y.double().cpu().numpy())
    assert rep["rel_kkt"] <= REL_KKT, rep
    assert abs(rep["rel_kkt"] - res["kkt"]["rel_kkt"]) <= 1e-7 + 1e-3 * rep["rel_kkt"]
    assert abs(rep["pobj"] - res["kkt"]["pobj"]) <= 1e-6 * (1 + abs(rep["pobj"]))
    ref = _golden("socp_mix_objective.txt")    # the oracle's tol-1e-7 solve of the same instance
    assert ref["status"] == 0 and ref["rel_kkt"] <= 1e-7
    assert obj_close(rep["pobj"], ref["pobj"]), (rep["pobj"], ref["pobj"])


def test_socp_mix_full_spmv(gpu, orc, socp):
    import torch
    m, n = socp["m"], socp["n"]
    rp, ci = socp["a_rowptr"], socp["a_colind"]
    x = np.random.default_rng(71).normal(size=n)
    vt = torch.tensor(socp["a_val"], dtype=torch.float32, device="cuda")
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    yt = torch.zeros(m, dtype=torch.float32, device="cuda")
    rpt = torch.tensor(rp, dtype=torch.int32, device="cuda")
    cit = torch.tensor(ci, dtype=torch.int32, device="cuda")
    gpu.cqp_spmv(0, m, n, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(), xt.data_ptr(), yt.data_ptr(), 0)
    vr, xr = vt.double().cpu().numpy(), xt.double().cpu().numpy()
    ref = orc.spmv(rp, ci, vr, xr)
    scale = orc.spmv(rp, ci, np.abs(vr), np.abs(xr)) + 1e-300
    assert (np.abs(yt.double().cpu().numpy() - ref) / scale).max() <= 1e-5


def _project_sampled(gpu, orc, inst, metric, kinds, nsample, seed):
    """Project the instance's full cone layout on the GPU (FP32) and check sampled blocks of the
    given kinds against the oracle's FP64 projection of the same FP32 inputs."""
    import torch
    rng = np.random.default_rng(seed)
    n = inst["n"]
    types, starts, dims, alphas = inst["blk_type"], inst["blk_start"], inst["blk_dim"], inst["blk_alpha"]
    r = rng.normal(size=n) * np.repeat(10.0 ** rng.uniform(-2, 2, size=types.size), dims)
    rt = torch.tensor(r, dtype=torch.float32, device="cuda")
    mt = torch.tensor(np.exp(rng.normal(size=n) * 0.7), dtype=torch.float32, device="cuda") if metric else None
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    dev = [torch.tensor(np.ascontiguousarray(a), device="cuda") for a in
           (types.astype(np.int32), starts.astype(np.int64), dims.astype(np.int64), alphas.astype(np.float64))]
    K = gpu.Cones(types.size, *[a.data_ptr() for a in dev])
    gpu.cqp_project(0, n, K, rt.data_ptr(), None if mt is None else mt.data_ptr(), out.data_ptr())
    got, rr = out.double().cpu().numpy(), rt.double().cpu().numpy()
    mm = None if mt is None else mt.double().cpu().numpy()
    cand = np.nonzero(np.isin(types, kinds))[0]
    pick = rng.choice(cand, size=min(nsample, cand.size), replace=False)
    for j in pick:
        t, s, d, a = int(types[j]), int(starts[j]), int(dims[j]), float(alphas[j])
        ref = orc.proj_block(t, rr[s:s + d], alpha=a, m=None if mm is None else mm[s:s + d])
        assert np.abs(got[s:s + d] - ref).max() <= 1e-5 * (1.0 + np.abs(rr[s:s + d]).max()), (t, d)
    return pick.size


@pytest.mark.parametrize("metric", [False, True])
def test_socp_mix_full_projections(gpu, orc, socp, metric):
    assert _project_sampled(gpu, orc, socp, metric, (G.SOC, G.RSOC), 300, 72 + metric) == 300


@pytest.mark.parametrize("metric", [False, True])
@pytest.mark.parametrize("fixed_middle", [True, False])
def test_fisher_full_projections(gpu, orc, metric, fixed_middle):
    inst = I.fisher_market(fixed_middle=fixed_middle)
    kinds = (G.EXP1, G.POW1) if fixed_middle else (G.EXP, G.POW)
    assert _project_sampled(gpu, orc, inst, metric, kinds, 400, 74 + metric) == 400


def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = float(v)
    return vals


@pytest.fixture(scope="module")
def fisher():
    return I.fisher_market()


@pytest.mark.parametrize("precision", [0, 1])
def test_fisher_full_solve(gpu, orc, fisher, precision):
    """Full Fisher market (reading D24 slices) to rel-KKT <= 1e-4 in FP32 iterates and in FP64."""
    ref = _golden("fisher_10000x1000_objective.txt")    # the oracle's tol-1e-7 solve
    assert ref["status"] == 0 and ref["rel_kkt"] <= 1e-7
    s = gpu.Solver(_device(fisher), precision=precision, tol=1e-4, max_iter=400000, time_limit_s=300.0)
    x, y, res = s.solve(out_device=True)
    s.close()
    assert res["rc"] == 0, res
    rep = orc.kkt(fisher, x.double().cpu().numpy(), y.double().cpu().numpy())
    assert rep["rel_kkt"] <= REL_KKT, rep
    assert obj_close(rep["pobj"], ref["pobj"]), (rep["pobj"], ref["pobj"])


def test_portfolio_full_batch_sampled(gpu, orc):
    batch = I.portfolio_batch()
    s = gpu.BatchSolver(batch, precision=0, tol=1e-4, max_iter=200000, time_limit_s=600.0)
    x, y, per, res = s.solve()
    s.close()
    assert res["rc"] == 0, res
    assert len(per) == batch["batch_count"] == 4096
    assert all(r["rc"] == 0 for r in per)
    rng = np.random.default_rng(76)
    for i in rng.choice(4096, size=16, replace=False):
        member = I.batch_member(batch, int(i))
        x0, x1 = int(batch["x_off"][i]), int(batch["x_off"][i + 1])
        r0, r1 = int(batch["row_off"][i]), int(batch["row_off"][i + 1])
        rep = orc.kkt(member, x[x0:x1], y[r0:r1])
        assert rep["rel_kkt"] <= REL_KKT, (i, rep)
        assert abs(rep["rel_kkt"] - per[i]["kkt"]["rel_kkt"]) <= 1e-7 + 1e-3 * rep["rel_kkt"], i
        _, _, info = orc.solve(member, max_iter=1000000, tol=1e-9)
        assert obj_close(rep["pobj"], info["kkt"]["pobj"]), (i, rep["pobj"], info["kkt"]["pobj"])


def test_qcqp_frontend_full(gpu, orc):
    from paper_2608_09159_gb300 import frontends as F
    Q = I.qcqp_problem(n=200_000, m_lin=50_000, p=50, k=50, k0=20, c_nnz=2000)
    inst, _ = F.qcqp_to_qsocp(Q["n"], Q["c0"], Q["quad"], q0_diag=Q["q0_diag"], q0_R=Q["q0_R"], A=Q["A"],
                              row_lo=Q["row_lo"], row_hi=Q["row_hi"], x_lo=Q["x_lo"], x_hi=Q["x_hi"])
    s = gpu.Solver(_device(inst), precision=0, tol=1e-4, max_iter=200000, time_limit_s=600.0)
    x, y, res = s.solve(out_device=True)
    s.close()
    assert res["rc"] == 0, res
    rep = orc.kkt(inst, x.double().cpu().numpy(), y.double().cpu().numpy())
    assert rep["rel_kkt"] <= REL_KKT, rep
    assert abs(rep["rel_kkt"] - res["kkt"]["rel_kkt"]) <= 1e-7 + 1e-3 * rep["rel_kkt"]
