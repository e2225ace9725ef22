"""Host logic of the library's modeling front-ends (paper_2608_09159_gb300/frontends.py) on
cases the oracle-equality test does not reach, solved by the oracle (no GPU):
* a QCQP with no linear rows and no bounds: a free block, one RSOC block per constraint, and
  the ball closed form x* = -sqrt(2d) c/||c||;
* a sparse P part of Q0 extended to the lifted variables (Q products equal the dense Q0);
* a constraint with a zero-row factor is rejected;
* the Lasso with A = I: rows, Q, c as specified and x* = soft(b, lam/2).
"""
import numpy as np
import pytest

from paper_2608_09159_gb300 import frontends as F


def _csr(M):
    rows, cols = np.nonzero(M)
    rp = np.zeros(M.shape[0] + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols.astype(np.int64), M[rows, cols]


def test_qcqp_without_rows_or_bounds(orc):
    rng = np.random.default_rng(101)
    n, d = 6, 0.4
    c0 = rng.normal(size=n)
    quad = [dict(R=_csr(np.eye(n)), k=n, c=None, d=d)]
    inst, rec = F.qcqp_to_qsocp(n, c0, quad)
    assert list(inst["blk_type"]) == [F.FREE, F.RSOC] and list(inst["blk_dim"]) == [n, n + 2]
    assert inst["m"] == n + 2 and "x_lo" not in inst
    x, y, info = orc.solve(inst, tol=1e-9, max_iter=200000)
    assert info["status"] == 0
    assert np.abs(rec(x) + np.sqrt(2 * d) * c0 / np.linalg.norm(c0)).max() <= 1e-6


def test_qcqp_sparse_q0_is_extended(orc):
    rng = np.random.default_rng(102)
    n = 8
    M = rng.normal(size=(n, n)) * (rng.uniform(size=(n, n)) < 0.4)
    P = M @ M.T
    quad = [dict(R=_csr(rng.normal(size=(3, n))), k=3, c=rng.normal(size=n), d=5.0)]
    inst, rec = F.qcqp_to_qsocp(n, rng.normal(size=n), quad, q0_diag=np.ones(n), q0_P=_csr(P))
    N = inst["n"]
    z = rng.normal(size=N)
    ref = np.zeros(N)
    ref[:n] = (np.eye(n) + P) @ z[:n]
    assert np.allclose(orc.q_apply(inst, z), ref, rtol=1e-13, atol=1e-12)


def test_qcqp_rejects_empty_factor():
    with pytest.raises(ValueError):
        F.qcqp_to_qsocp(3, np.zeros(3), [dict(R=(np.zeros(1, np.int64), np.zeros(0, np.int64), np.zeros(0)), k=0,
                                              c=None, d=1.0)])


def test_lasso_identity(orc):
    rng = np.random.default_rng(103)
    n, lam = 10, 0.6
    b = rng.normal(size=n)
    inst, rec = F.lasso_to_qp(_csr(np.eye(n)), b, lam, m=n, n=n)
    assert inst["m"] == n + 2 * n and inst["n"] == 3 * n
    assert np.array_equal(inst["q_diag"], np.concatenate([np.zeros(n), 2 * np.ones(n), np.zeros(n)]))
    assert np.array_equal(inst["c"], np.concatenate([np.zeros(2 * n), lam * np.ones(n)]))
    x, y, info = orc.solve(inst, tol=1e-10, max_iter=400000)
    assert info["status"] == 0
    ref = np.sign(b) * np.maximum(np.abs(b) - lam / 2, 0.0)
    assert np.abs(rec(x) - ref).max() <= 1e-6
