"""Pins of the oracle's general form (Sec. 4 standard form): row bounds lo <= Ax <= hi and
box blocks lo <= x <= hi.

* a box-constrained QP with diagonal Q has the closed form x = clip(-c/q, lo, hi);
* inequality rows give the same optimum as the equality form with box-bounded slacks
  (a reformulation handled entirely by the already-pinned equality path);
* an LP with two-sided rows and boxes matches scipy's linprog;
* the KKT report vanishes at the optimum and not at a perturbed point.
"""
import numpy as np
import pytest

import instances as I

BOX = 6


def _inst(A, c, blocks, q=None, b=None, lo=None, hi=None, xlo=None, xhi=None):
    m, n = A.shape
    r, cidx = np.nonzero(A)
    rp, ci, v = I._coo_to_csr(m, n, r, cidx, A[r, cidx])
    bt, bs, bd, ba = I.blocks_from_list(blocks)
    inst = I.make_instance("t", m, n, rp, ci, v, c, np.zeros(m) if b is None else b, bt, bs, bd, ba, q_diag=q)
    if lo is not None:
        inst["row_lo"], inst["row_hi"] = np.asarray(lo, float), np.asarray(hi, float)
    if xlo is not None:
        inst["x_lo"], inst["x_hi"] = np.asarray(xlo, float), np.asarray(xhi, float)
    return inst


def test_box_qp_closed_form(orc):
    rng = np.random.default_rng(11)
    n = 40
    q = rng.uniform(0.5, 2.0, n)
    c = rng.normal(size=n) * 2
    lo = rng.uniform(-1.0, 0.0, n)
    hi = rng.uniform(0.0, 1.0, n)
    lo[:5] = -np.inf
    hi[5:10] = np.inf
    # one free coordinate z with the row z = 0 keeps the problem in standard form
    A = np.zeros((1, n + 1))
    A[0, n] = 1.0
    inst = _inst(A, np.concatenate([c, [0.0]]), [(BOX, n, 0.0), (I.CONE_FREE, 1, 0.0)],
                 q=np.concatenate([q, [1.0]]), b=np.zeros(1),
                 xlo=np.concatenate([lo, [0.0]]), xhi=np.concatenate([hi, [0.0]]))
    x, y, info = orc.solve(inst, max_iter=200000, tol=1e-10)
    ref = np.clip(-c / q, lo, hi)
    assert np.abs(x[:n] - ref).max() <= 1e-7
    assert info["kkt"]["rel_kkt"] <= 1e-9


def _random_rows(rng, m, n):
    A = rng.normal(size=(m, n)) * (rng.uniform(size=(m, n)) < 0.4)
    for i in range(m):
        if not A[i].any():
            A[i, rng.integers(n)] = 1.0
    return A


def test_inequality_rows_equal_slack_form(orc):
    rng = np.random.default_rng(12)
    m, n = 12, 25
    A = _random_rows(rng, m, n)
    x0 = np.abs(rng.normal(size=n))
    ax0 = A @ x0
    lo = ax0 - rng.uniform(0.1, 1.0, m)
    hi = ax0 + rng.uniform(0.1, 1.0, m)
    lo[:3] = hi[:3] = ax0[:3]        # equality rows
    lo[3:6] = -np.inf                # one-sided rows
    hi[6:8] = np.inf
    q = rng.uniform(0.2, 1.0, n)
    c = rng.normal(size=n)
    ineq = _inst(A, c, [(I.CONE_NONNEG, n, 0.0)], q=q, lo=lo, hi=hi)
    x1, y1, i1 = orc.solve(ineq, max_iter=400000, tol=1e-9)
    # slack form: A x - s = 0, s in box [lo, hi]
    As = np.hstack([A, -np.eye(m)])
    slack = _inst(As, np.concatenate([c, np.zeros(m)]), [(I.CONE_NONNEG, n, 0.0), (BOX, m, 0.0)],
                  q=np.concatenate([q, np.zeros(m)]), b=np.zeros(m),
                  xlo=np.concatenate([np.zeros(n), lo]), xhi=np.concatenate([np.zeros(n), hi]))
    x2, y2, i2 = orc.solve(slack, max_iter=400000, tol=1e-9)
    assert np.abs(x1 - x2[:n]).max() <= 1e-5 * (1 + np.abs(x2).max())
    assert abs(i1["kkt"]["pobj"] - i2["kkt"]["pobj"]) <= 1e-7 * (1 + abs(i2["kkt"]["pobj"]))


def test_lp_matches_linprog(orc):
    linprog = pytest.importorskip("scipy.optimize").linprog
    rng = np.random.default_rng(13)
    m, n = 10, 20
    A = _random_rows(rng, m, n)
    x0 = rng.uniform(-0.5, 1.5, n)
    ax0 = A @ x0
    lo = ax0 - rng.uniform(0.1, 0.5, m)
    hi = ax0 + rng.uniform(0.1, 0.5, m)
    hi[:3] = np.inf
    c = rng.normal(size=n)
    xlo, xhi = np.full(n, -1.0), np.full(n, 2.0)
    inst = _inst(A, c, [(BOX, n, 0.0)], lo=lo, hi=hi, xlo=xlo, xhi=xhi)
    x, y, info = orc.solve(inst, max_iter=1000000, tol=1e-8)
    fin = np.isfinite(hi)
    ref = linprog(c, A_ub=np.vstack([A[fin], -A]), b_ub=np.concatenate([hi[fin], -lo]),
                  bounds=list(zip(xlo, xhi)), method="highs")
    assert ref.status == 0
    assert abs(c @ x - ref.fun) <= 1e-5 * (1 + abs(ref.fun))
    rep = orc.kkt(inst, x, y)
    assert rep["rel_kkt"] <= 1e-7
    bad = orc.kkt(inst, x + 0.01, y)
    assert bad["rel_kkt"] > 1e-4
