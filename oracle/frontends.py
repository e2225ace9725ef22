"""Oracle-side reformulations for the modeling front-ends. TEST INFRASTRUCTURE ONLY: used by
the test suite to check the library's front-ends; shares no code with them.

Written plainly with dense matrices (small sizes only), straight from the paper:
* QCQP (eq. qcqp-benchmark-form) to QSOCP: each 1/2 x'R'R x + c'x <= d becomes
  (d - c'x, 1, R x) in K_rsoc (eq. qcqp-to-rsoc). In the (v, s, t) order of the oracle's RSOC
  ({||v||^2 <= 2 s t}) that is v = R x, s = 1, t = d - c'x. Here those are new variables tied
  to x by equality rows.
* Lasso to QP (Sec. 5.5): min y'y + lam 1't s.t. y = Ax - b, -t <= x <= t.
The problems are plain (x, y) dicts for ``oracle.solve``; the first n coordinates of x are
the original variables.
"""
from __future__ import annotations

import numpy as np

FREE, NONNEG, SOC, RSOC, EXP, POW, BOX = 0, 1, 2, 3, 4, 5, 6


def _dense(csr, nrows, ncols):
    rp, ci, v = csr
    M = np.zeros((nrows, ncols))
    for i in range(nrows):
        for t in range(int(rp[i]), int(rp[i + 1])):
            M[i, int(ci[t])] += v[t]
    return M


def _instance(name, Aeq, lo, hi, c, blocks, q_diag=None, P=None, xlo=None, xhi=None):
    m, N = Aeq.shape
    rows, cols = np.nonzero(Aeq)
    rowptr = np.zeros(m + 1, np.int64)
    for r in rows:
        rowptr[r + 1] += 1
    rowptr = np.cumsum(rowptr)
    bt = np.array([b[0] for b in blocks], np.int32)
    bd = np.array([b[1] for b in blocks], np.int64)
    bs = np.concatenate([[0], np.cumsum(bd)[:-1]]).astype(np.int64)
    inst = dict(name=name, m=m, n=N, a_rowptr=rowptr, a_colind=cols.astype(np.int64), a_val=Aeq[rows, cols],
                c=np.asarray(c, float), b=np.zeros(m), row_lo=np.asarray(lo, float), row_hi=np.asarray(hi, float),
                blk_type=bt, blk_start=bs, blk_dim=bd, blk_alpha=np.zeros(bd.size),
                q_diag=None if q_diag is None else np.asarray(q_diag, float))
    if P is not None:
        pr, pc = np.nonzero(P)
        prp = np.zeros(N + 1, np.int64)
        for r in pr:
            prp[r + 1] += 1
        inst["p_rowptr"], inst["p_colind"], inst["p_val"] = np.cumsum(prp), pc.astype(np.int64), P[pr, pc]
    if xlo is not None:
        inst["x_lo"], inst["x_hi"] = np.asarray(xlo, float), np.asarray(xhi, float)
    return inst


def qcqp(prob):
    """QSOCP form of an instances.qcqp_problem dict: Q0 kept in the objective as a dense P
    (diag + R0'R0), one RSOC block per quadratic constraint."""
    n = prob["n"]
    quad = prob["quad"]
    N = n + sum(q["k"] + 2 for q in quad)
    Q0 = np.diag(prob["q0_diag"]) + prob["q0_R"].T @ prob["q0_R"]
    P = np.zeros((N, N))
    P[:n, :n] = Q0
    rows, lo, hi = [], [], []
    A = _dense(prob["A"], prob["m_lin"], n)
    for i in range(prob["m_lin"]):
        r = np.zeros(N)
        r[:n] = A[i]
        rows.append(r); lo.append(prob["row_lo"][i]); hi.append(prob["row_hi"][i])
    off = n
    blocks = [(BOX, n)]
    for q in quad:
        k = q["k"]
        R = _dense(q["R"], k, n)
        for j in range(k):            # v_j = (R x)_j
            r = np.zeros(N)
            r[:n] = R[j]
            r[off + j] = -1.0
            rows.append(r); lo.append(0.0); hi.append(0.0)
        r = np.zeros(N)               # s = 1
        r[off + k] = 1.0
        rows.append(r); lo.append(1.0); hi.append(1.0)
        r = np.zeros(N)               # t = d - c'x
        r[:n] = q["c"]
        r[off + k + 1] = 1.0
        rows.append(r); lo.append(q["d"]); hi.append(q["d"])
        blocks.append((RSOC, k + 2))
        off += k + 2
    xlo = np.full(N, -np.inf)
    xhi = np.full(N, np.inf)
    xlo[:n], xhi[:n] = prob["x_lo"], prob["x_hi"]
    c = np.zeros(N)
    c[:n] = prob["c0"]
    return _instance("qcqp_oracle", np.array(rows), lo, hi, c, blocks, P=P, xlo=xlo, xhi=xhi)


def qcqp_objective(prob, x):
    Q0x = prob["q0_diag"] * x + prob["q0_R"].T @ (prob["q0_R"] @ x)
    return 0.5 * x @ Q0x + prob["c0"] @ x


def lasso(A, b, lam):
    """QP form of the Lasso with dense A (m x n)."""
    m, n = A.shape
    N = n + m + n
    rows, lo, hi = [], [], []
    for i in range(m):                # y_i - (A x)_i = -b_i
        r = np.zeros(N)
        r[:n] = -A[i]
        r[n + i] = 1.0
        rows.append(r); lo.append(-b[i]); hi.append(-b[i])
    for j in range(n):                # x_j - t_j <= 0
        r = np.zeros(N)
        r[j] = 1.0
        r[n + m + j] = -1.0
        rows.append(r); lo.append(-np.inf); hi.append(0.0)
    for j in range(n):                # x_j + t_j >= 0
        r = np.zeros(N)
        r[j] = 1.0
        r[n + m + j] = 1.0
        rows.append(r); lo.append(0.0); hi.append(np.inf)
    q = np.zeros(N)
    q[n:n + m] = 2.0                  # y'y = 1/2 y'(2I)y
    c = np.zeros(N)
    c[n + m:] = lam
    return _instance("lasso_oracle", np.array(rows), lo, hi, c, [(FREE, N)], q_diag=q)


def lasso_objective(A, b, lam, x):
    r = A @ x - b
    return r @ r + lam * np.abs(x).sum()
