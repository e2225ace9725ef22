"""GPU parity of problems built by the modeling front-ends (paper_2608_09159_gb300/frontends.py).

Each front-end instance is solved through cqp_setup_general on the GPU in FP32 and FP64.
* The returned point reaches rel-KKT <= 1e-4, re-measured by the oracle on the same
  instance.
* The original problem's objective at the recovered x matches the oracle's solve of its own
  reformulation (oracle/frontends.py), written independently.
* x matches the oracle's tight solution, which is unique for these instances: Q0 is
  positive definite for the QCQP, and A has full column rank for the Lasso.
"""
import numpy as np
import pytest

from _parity import REL_KKT, obj_close

import instances as I
from oracle import frontends as OF

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


@pytest.fixture(scope="module")
def qcqp_case(orc):
    prob = I.qcqp_problem(n=300, m_lin=60, p=4, k=8, k0=5, lin_per_row=6, quad_per_row=6, seed=61)
    xo, yo, info = orc.solve(OF.qcqp(prob), tol=1e-8, max_iter=400000)
    assert info["status"] == 0
    return prob, xo[:prob["n"]]


@pytest.mark.parametrize("precision", [1, 0])
def test_qcqp_frontend(gpu, orc, qcqp_case, precision):
    from paper_2608_09159_gb300 import frontends as F
    prob, xref = qcqp_case
    inst, rec = F.qcqp_to_qsocp(prob["n"], prob["c0"], prob["quad"], q0_diag=prob["q0_diag"], q0_R=prob["q0_R"],
                                A=prob["A"], row_lo=prob["row_lo"], row_hi=prob["row_hi"], x_lo=prob["x_lo"],
                                x_hi=prob["x_hi"])
    s = gpu.Solver(inst, precision=precision, tol=1e-4, max_iter=200000, time_limit_s=120.0)
    x, y, res = s.solve()
    s.close()
    assert res["rc"] == 0, res
    rep = orc.kkt(inst, x, y)
    assert rep["rel_kkt"] <= REL_KKT, rep
    xs = rec(x)
    assert obj_close(OF.qcqp_objective(prob, xs), OF.qcqp_objective(prob, xref))
    assert np.linalg.norm(xs - xref) <= 2e-2 * (1 + np.linalg.norm(xref))


@pytest.fixture(scope="module")
def lasso_case(orc):
    L = I.lasso_problem(m=400, n=120, density=0.05, seed=62)
    A = OF._dense((L["a_rowptr"], L["a_colind"], L["a_val"]), L["m"], L["n"])
    xo, yo, info = orc.solve(OF.lasso(A, L["b"], L["lam"]), tol=1e-9, max_iter=400000)
    assert info["status"] == 0
    return L, A, xo[:L["n"]]


@pytest.mark.parametrize("precision", [1, 0])
def test_lasso_frontend(gpu, orc, lasso_case, precision):
    from paper_2608_09159_gb300 import frontends as F
    L, A, xref = lasso_case
    inst, rec = F.lasso_to_qp((L["a_rowptr"], L["a_colind"], L["a_val"]), L["b"], L["lam"], m=L["m"], n=L["n"])
    s = gpu.Solver(inst, precision=precision, tol=1e-4, max_iter=200000, time_limit_s=120.0)
    x, y, res = s.solve()
    s.close()
    assert res["rc"] == 0, res
    rep = orc.kkt(inst, x, y)
    assert rep["rel_kkt"] <= REL_KKT, rep
    xs = rec(x)
    f, fref = OF.lasso_objective(A, L["b"], L["lam"], xs), OF.lasso_objective(A, L["b"], L["lam"], xref)
    assert obj_close(f, fref), (f, fref)
    assert np.linalg.norm(xs - xref) <= 2e-2 * (1 + np.linalg.norm(xref))
