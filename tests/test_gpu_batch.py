"""GPU parity of the batched persistent solve (cqp_setup_batch / cqp_solve_batch).

A batch of small portfolio QPs (config 4 at oracle scale) is solved in one
launch.  Each instance must:

* reach rel-KKT <= 1e-4 as re-measured by the CPU oracle on the instance alone;
* agree in objective with the oracle's own solve of that instance;
* have the oracle's x where x is unique (Q = D + FF' is positive definite on x);
* match the single-instance GPU solve of the same data.

Malformed batches are rejected before any solve.
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


def _rel(a, b):
    return abs(a - b) / (1.0 + abs(a) + abs(b))


def _slices(inst, i):
    return (slice(int(inst["x_off"][i]), int(inst["x_off"][i + 1])),
            slice(int(inst["row_off"][i]), int(inst["row_off"][i + 1])))


@pytest.mark.parametrize("precision", [1, 0])
def test_batch_instances_match_oracle(gpu, orc, precision):
    batch = I.small_config(4)
    s = gpu.BatchSolver(batch, precision=precision, tol=1e-4, max_iter=200000, time_limit_s=120.0)
    x, y, per, res = s.solve()
    s.close()
    assert res["rc"] == 0, res
    assert len(per) == batch["batch_count"]
    for i, r in enumerate(per):
        assert r["rc"] == 0, (i, r)
        member = I.batch_member(batch, i)
        xs, ys = _slices(batch, i)
        rep = orc.kkt(member, x[xs], y[ys])
        assert rep["rel_kkt"] <= REL_KKT, (i, rep)
        assert abs(rep["rel_kkt"] - r["kkt"]["rel_kkt"]) <= 1e-7 + 1e-3 * rep["rel_kkt"], (i, rep, r)
        xt, yt, info = orc.solve(member, max_iter=1000000, tol=TIGHT_TOL)
        assert obj_close(rep["pobj"], info["kkt"]["pobj"]), (i, rep["pobj"], info["kkt"]["pobj"])
        na = int(batch["n_assets"][i])
        assert np.linalg.norm(x[xs][:na] - xt[:na]) <= 2e-2 * (1 + np.linalg.norm(xt[:na])), i


def test_batch_equals_single_instance_solves(gpu):
    # same arithmetic per instance: scaling, step sizes and stop test as if solved alone
    batch = I.small_config(4)
    opts = dict(precision=1, tol=1e-4, max_iter=200000, time_limit_s=120.0, tpr_a=4, tpr_at=4)
    s = gpu.BatchSolver(batch, **opts)
    x, y, per, res = s.solve()
    s.close()
    for i in range(batch["batch_count"]):
        member = I.batch_member(batch, i)
        t = gpu.Solver(member, team=2, **opts)
        xm, ym, rm = t.solve()
        t.close()
        assert rm["rc"] == 0
        xs, ys = _slices(batch, i)
        assert abs(per[i]["iters"] - rm["iters"]) <= 2 * 64, (i, per[i]["iters"], rm["iters"])
        assert _rel(per[i]["kkt"]["pobj"], rm["kkt"]["pobj"]) <= 1e-4, i
        assert np.abs(x[xs] - xm).max() <= 5e-3 * (1 + np.abs(xm).max()), i


def test_batch_warm_start_from_solution(gpu, orc):
    batch = I.small_config(4)
    x0 = np.zeros(batch["n"])
    y0 = np.zeros(batch["m"])
    for i in range(batch["batch_count"]):
        xs, ys = _slices(batch, i)
        xt, yt, _ = orc.solve(I.batch_member(batch, i), max_iter=400000, tol=1e-7)
        x0[xs], y0[ys] = xt, yt
    s = gpu.BatchSolver(batch, precision=1, tol=1e-4, max_iter=200000, time_limit_s=60.0)
    x, y, per, res = s.solve(x0=x0, y0=y0)
    s.close()
    assert res["rc"] == 0
    assert max(r["iters"] for r in per) <= 128


def test_batch_invalid_inputs(gpu):
    batch = I.small_config(4)
    bad = dict(batch)
    bad["x_off"] = batch["x_off"].copy()
    bad["x_off"][1] += 1                       # a cone block now straddles instances 0 and 1
    with pytest.raises(gpu.CQPError) as e:
        gpu.BatchSolver(bad)
    assert e.value.code == -1
    bad = dict(batch)
    bad["row_off"] = batch["row_off"].copy()
    bad["row_off"][1] -= 1                     # a row of instance 0 is assigned to instance 1
    with pytest.raises(gpu.CQPError) as e:
        gpu.BatchSolver(bad)
    assert e.value.code == -1
    bad = dict(batch)
    bad["x_off"] = batch["x_off"].copy()
    bad["x_off"][-1] -= 1                      # offsets do not end at n
    with pytest.raises(gpu.CQPError) as e:
        gpu.BatchSolver(bad)
    assert e.value.code == -1
    # a single-problem handle refuses the batch entry point and vice versa
    s = gpu.Solver(I.batch_member(batch, 0))
    with pytest.raises(gpu.CQPError):
        gpu.cqp_solve_batch(s.h, None, None, None, None, 0, None, gpu.Result())
    s.close()
