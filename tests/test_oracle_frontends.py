"""Pins of the modeling front-ends (Sec. 5.3 QCQP -> QSOCP by eq. qcqp-to-rsoc, Sec. 5.5 Lasso -> QP).

Oracle side (oracle/frontends.py + oracle.solve) against facts about the ORIGINAL problems:
* min c'x s.t. 1/2||x||^2 <= d has x* = -sqrt(2d) c/||c||;
* min 1/2||x - p||^2 s.t. 1/2||x||^2 <= d (active) has x* = p sqrt(2d)/||p||;
* a small random convex QCQP matches scipy's SLSQP on the original form;
* the Lasso with A = I has x* = soft(b, lam/2);
* a small random Lasso meets its subgradient optimality conditions and matches scikit-learn.
Host logic of the library's front-end (paper_2608_09159_gb300/frontends.py, no GPU):
* it builds the same rows, bounds, cones, c and Q as the oracle's plain restatement.
"""
import numpy as np
import pytest

import instances as I
from oracle import frontends as OF
from paper_2608_09159_gb300 import frontends as PF


def _csr_dense(mat):
    rows, cols = np.nonzero(mat)
    rp = np.zeros(mat.shape[0] + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols.astype(np.int64), mat[rows, cols]


def _qcqp_prob(n, c0, q0_diag, R0, quad, A=None, lo=None, hi=None, box=np.inf):
    m_lin = 0 if A is None else A.shape[0]
    Acsr = _csr_dense(A if A is not None else np.zeros((0, n)))
    return dict(n=n, c0=np.asarray(c0, float), q0_diag=np.asarray(q0_diag, float), q0_R=np.asarray(R0, float),
                A=Acsr, m_lin=m_lin, row_lo=np.zeros(0) if lo is None else lo,
                row_hi=np.zeros(0) if hi is None else hi, x_lo=np.full(n, -box), x_hi=np.full(n, box),
                quad=[dict(R=_csr_dense(R), k=R.shape[0], c=np.asarray(c, float), d=float(d)) for R, c, d in quad])


def test_linear_objective_over_ball(orc):
    rng = np.random.default_rng(51)
    n, d = 8, 0.7
    c0 = rng.normal(size=n)
    prob = _qcqp_prob(n, c0, np.zeros(n), np.zeros((1, n)), [(np.eye(n), np.zeros(n), d)])
    x, y, info = orc.solve(OF.qcqp(prob), tol=1e-9, max_iter=200000)
    assert info["status"] == 0
    ref = -np.sqrt(2 * d) * c0 / np.linalg.norm(c0)
    assert np.abs(x[:n] - ref).max() <= 1e-6


def test_projection_onto_ball(orc):
    rng = np.random.default_rng(52)
    n, d = 8, 0.3
    p = rng.normal(size=n) * 2
    prob = _qcqp_prob(n, -p, np.ones(n), np.zeros((1, n)), [(np.eye(n), np.zeros(n), d)])
    x, y, info = orc.solve(OF.qcqp(prob), tol=1e-9, max_iter=200000)
    assert info["status"] == 0
    ref = p * np.sqrt(2 * d) / np.linalg.norm(p)
    assert np.abs(x[:n] - ref).max() <= 1e-6


def test_random_qcqp_matches_slsqp(orc):
    minimize = pytest.importorskip("scipy.optimize").minimize
    prob = I.qcqp_problem(n=10, m_lin=3, p=2, k=3, k0=2, lin_per_row=4, quad_per_row=4, seed=53)
    x, y, info = orc.solve(OF.qcqp(prob), tol=1e-10, max_iter=400000)
    assert info["status"] == 0
    n = prob["n"]
    A = OF._dense(prob["A"], prob["m_lin"], n)
    cons = []
    for i in range(prob["m_lin"]):
        if np.isfinite(prob["row_lo"][i]):
            cons.append(dict(type="ineq", fun=lambda z, i=i: A[i] @ z - prob["row_lo"][i], jac=lambda z, i=i: A[i]))
        cons.append(dict(type="ineq", fun=lambda z, i=i: prob["row_hi"][i] - A[i] @ z, jac=lambda z, i=i: -A[i]))
    for q in prob["quad"]:
        R = OF._dense(q["R"], q["k"], n)
        cons.append(dict(type="ineq", fun=lambda z, R=R, q=q: q["d"] - 0.5 * (R @ z) @ (R @ z) - q["c"] @ z,
                         jac=lambda z, R=R, q=q: -(R.T @ (R @ z)) - q["c"]))
    Q0 = np.diag(prob["q0_diag"]) + prob["q0_R"].T @ prob["q0_R"]
    res = minimize(lambda z: OF.qcqp_objective(prob, z), prob["x_feasible"], jac=lambda z: Q0 @ z + prob["c0"],
                   constraints=cons, bounds=list(zip(prob["x_lo"], prob["x_hi"])), method="SLSQP",
                   options=dict(ftol=1e-14, maxiter=2000))
    assert res.success
    f_orc = OF.qcqp_objective(prob, x[:n])
    assert abs(f_orc - res.fun) <= 1e-6 * (1 + abs(res.fun))
    assert np.abs(x[:n] - res.x).max() <= 1e-4          # Q0 positive definite: x* unique


def test_lasso_identity_soft_threshold(orc):
    rng = np.random.default_rng(54)
    n, lam = 12, 0.8
    b = rng.normal(size=n)
    x, y, info = orc.solve(OF.lasso(np.eye(n), b, lam), tol=1e-10, max_iter=400000)
    assert info["status"] == 0
    ref = np.sign(b) * np.maximum(np.abs(b) - lam / 2, 0.0)
    assert np.abs(x[:n] - ref).max() <= 1e-6


def _lasso_small(seed):
    L = I.lasso_problem(m=40, n=15, density=0.3, seed=seed)
    A = OF._dense((L["a_rowptr"], L["a_colind"], L["a_val"]), L["m"], L["n"])
    return L, A


def test_lasso_subgradient_and_sklearn(orc):
    L, A = _lasso_small(55)
    b, lam, n = L["b"], L["lam"], L["n"]
    x, y, info = orc.solve(OF.lasso(A, b, lam), tol=1e-10, max_iter=400000)
    assert info["status"] == 0
    xs = x[:n]
    g = 2 * A.T @ (b - A @ xs)            # must lie in lam * subdifferential of ||x||_1
    nz = np.abs(xs) > 1e-7
    assert np.abs(g[nz] - lam * np.sign(xs[nz])).max() <= 1e-5 * (1 + lam)
    assert (np.abs(g[~nz]) <= lam * (1 + 1e-6) + 1e-6).all()
    sk = pytest.importorskip("sklearn.linear_model")
    ref = sk.Lasso(alpha=lam / (2 * A.shape[0]), fit_intercept=False, tol=1e-14, max_iter=1_000_000).fit(A, b).coef_
    assert abs(OF.lasso_objective(A, b, lam, xs) - OF.lasso_objective(A, b, lam, ref)) <= 1e-8 * (1 + abs(
        OF.lasso_objective(A, b, lam, ref)))
    assert np.abs(xs - ref).max() <= 1e-4


def _same_instance(orc, a, b):
    assert a["m"] == b["m"] and a["n"] == b["n"]
    rng = np.random.default_rng(0)
    for _ in range(3):
        z = rng.normal(size=a["n"])
        assert np.allclose(I.csr_matvec(a["a_rowptr"], a["a_colind"], a["a_val"], z),
                           I.csr_matvec(b["a_rowptr"], b["a_colind"], b["a_val"], z), rtol=1e-13, atol=1e-12)
        assert np.allclose(orc.q_apply(a, z), orc.q_apply(b, z), rtol=1e-12, atol=1e-12)
    for k in ("row_lo", "row_hi", "c", "blk_type", "blk_start", "blk_dim"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    for k in ("x_lo", "x_hi"):
        if k in a or k in b:
            assert np.array_equal(a[k], b[k]), k


def test_library_frontends_build_the_oracle_instances(orc):
    prob = I.qcqp_problem(n=30, m_lin=8, p=3, k=4, k0=3, lin_per_row=5, quad_per_row=5, seed=56)
    lib_inst, rec = PF.qcqp_to_qsocp(prob["n"], prob["c0"], prob["quad"], q0_diag=prob["q0_diag"], q0_R=prob["q0_R"],
                                     A=prob["A"], row_lo=prob["row_lo"], row_hi=prob["row_hi"], x_lo=prob["x_lo"],
                                     x_hi=prob["x_hi"])
    _same_instance(orc, lib_inst, OF.qcqp(prob))
    assert rec(np.arange(lib_inst["n"])).size == prob["n"]
    L, A = _lasso_small(57)
    lib_inst, rec = PF.lasso_to_qp((L["a_rowptr"], L["a_colind"], L["a_val"]), L["b"], L["lam"], m=L["m"], n=L["n"])
    _same_instance(orc, lib_inst, OF.lasso(A, L["b"], L["lam"]))
