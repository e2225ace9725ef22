"""Modeling front-ends: reformulations of two problem classes of the paper's experiments
into the solver's general standard form (Sec. 4, eq. solver-input).  Each returns an
instance dict that ``Solver`` accepts (it calls ``cqp_setup_general``) and a function that
recovers the original variables from the solver's x.

* ``qcqp_to_qsocp``: convex QCQP (eq. qcqp-benchmark-form) to a quadratic SOCP.  Q0 stays in
  the objective, and each quadratic constraint 1/2 x'R_i'R_i x + c_i'x <= d_i becomes a rotated
  second-order cone (d_i - c_i'x, 1, R_i x) in K_rsoc (eq. qcqp-to-rsoc).  The library's RSOC
  order is (v, s, t), with ||v||^2 <= 2 s t, so the block is (w_i, s_i, t_i) with
  w_i = R_i x, s_i = 1 and t_i = d_i - c_i'x.
* ``lasso_to_qp``: min ||Ax - b||^2 + lam ||x||_1 in the standard QP reformulation of
  Sec. 5.5, min y'y + lam 1't s.t. y = Ax - b, -t <= x <= t.

Host-side model building only: all solver arithmetic runs in the CUDA library.  Sparse
matrices are CSR triples (rowptr int64, colind int64, val float64).
"""
from __future__ import annotations

import numpy as np

FREE, NONNEG, SOC, RSOC, EXP, POW, BOX = 0, 1, 2, 3, 4, 5, 6


class _Rows:
    """Row-by-row CSR builder: append blocks of rows (as CSR pieces with a column offset)."""

    def __init__(self, ncols):
        self.ncols = ncols
        self.counts, self.cols, self.vals, self.lo, self.hi = [], [], [], [], []

    def add(self, rowptr, colind, val, lo, hi):
        rowptr = np.asarray(rowptr, np.int64)
        self.counts.append(np.diff(rowptr))
        self.cols.append(np.asarray(colind, np.int64))
        self.vals.append(np.asarray(val, np.float64))
        self.lo.append(np.broadcast_to(np.asarray(lo, np.float64), (rowptr.size - 1,)))
        self.hi.append(np.broadcast_to(np.asarray(hi, np.float64), (rowptr.size - 1,)))

    def csr(self):
        cnt = np.concatenate(self.counts) if self.counts else np.zeros(0, np.int64)
        rowptr = np.zeros(cnt.size + 1, np.int64)
        np.cumsum(cnt, out=rowptr[1:])
        cat = lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt)
        return rowptr, cat(self.cols, np.int64), cat(self.vals, np.float64), cat(self.lo, np.float64), \
            cat(self.hi, np.float64)


def _hstack_rows(parts, nrows):
    """Row-wise concatenation of CSR pieces [(rowptr, colind, val, col_offset), ...] with the same
    row count into one CSR."""
    counts = sum(np.diff(np.asarray(p[0], np.int64)) for p in parts)
    rowptr = np.zeros(nrows + 1, np.int64)
    np.cumsum(counts, out=rowptr[1:])
    cols = np.empty(rowptr[-1], np.int64)
    vals = np.empty(rowptr[-1], np.float64)
    fill = rowptr[:-1].copy()
    for rp, ci, v, off in parts:
        rp = np.asarray(rp, np.int64)
        cnt = np.diff(rp)
        row_of = np.repeat(np.arange(nrows, dtype=np.int64), cnt)
        pos = fill[row_of] + (np.arange(rp[-1], dtype=np.int64) - rp[:-1][row_of])
        cols[pos] = np.asarray(ci, np.int64) + off
        vals[pos] = v
        fill += cnt
    return rowptr, cols, vals


def _identity(n, scale=1.0):
    return np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int64), np.full(n, float(scale))


def _blocks(blist):
    t = np.array([b[0] for b in blist], np.int32)
    d = np.array([b[1] for b in blist], np.int64)
    s = np.zeros_like(d)
    if d.size:
        s[1:] = np.cumsum(d)[:-1]
    a = np.zeros(d.size)
    return t, s, d, a


def qcqp_to_qsocp(n, c0, quad, q0_diag=None, q0_R=None, q0_D=None, q0_P=None, A=None, row_lo=None, row_hi=None,
                  x_lo=None, x_hi=None, name="qcqp"):
    """Convex QCQP -> QSOCP instance (eqs. qcqp-benchmark-form, qcqp-to-rsoc).

    Objective 1/2 x'Q0 x + c0'x with Q0 = diag(q0_diag) + q0_P + q0_R' q0_D q0_R (any part may be
    None; q0_D defaults to I); linear rows row_lo <= A x <= row_hi (A a CSR triple with n
    columns, optional); bounds x_lo <= x <= x_hi (optional, infinite entries allowed); quad a
    sequence of dicts {"R": CSR triple with k rows and n columns, "k": k, "c": dense n or None,
    "d": float} meaning 1/2 ||R x||^2 + c'x <= d.

    Variables: [x | (w_1, s_1, t_1) | ... ], x one box (or free) block and one RSOC block per
    quadratic constraint.  Rows: the linear rows, then per constraint R_i x - w_i = 0,
    s_i = 1 and c_i'x + t_i = d_i.  Returns (instance, recover) with recover(x) -> x[:n].
    """
    c0 = np.asarray(c0, np.float64)
    ks = [int(q["k"]) for q in quad]
    if any(k < 1 for k in ks):
        raise ValueError("each quadratic constraint needs a factor with at least one row")
    N = n + sum(k + 2 for k in ks)
    rows = _Rows(N)
    if A is not None:
        rows.add(A[0], A[1], A[2], row_lo, row_hi)
    off = n
    for q, k in zip(quad, ks):
        rp, ci, v = q["R"]
        # R_i x - w_i = 0
        eye = _identity(k, -1.0)
        rows.add(*_hstack_rows([(rp, ci, v, 0), (eye[0], eye[1], eye[2], off)], k), 0.0, 0.0)
        # s_i = 1
        rows.add(np.array([0, 1]), np.array([off + k]), np.array([1.0]), 1.0, 1.0)
        # c_i'x + t_i = d_i
        c = np.zeros(n) if q.get("c") is None else np.asarray(q["c"], np.float64)
        nz = np.nonzero(c)[0]
        rows.add(np.array([0, nz.size + 1]), np.concatenate([nz, [off + k + 1]]), np.concatenate([c[nz], [1.0]]),
                 float(q["d"]), float(q["d"]))
        off += k + 2
    a_rp, a_ci, a_v, lo, hi = rows.csr()
    box = x_lo is not None or x_hi is not None
    blist = [(BOX if box else FREE, n)] + [(RSOC, k + 2) for k in ks]
    bt, bs, bd, ba = _blocks(blist)
    inst = dict(name=name, m=int(lo.size), n=int(N), a_rowptr=a_rp, a_colind=a_ci, a_val=a_v,
                c=np.concatenate([c0, np.zeros(N - n)]), b=np.zeros(lo.size), row_lo=lo, row_hi=hi,
                blk_type=bt, blk_start=bs, blk_dim=bd, blk_alpha=ba,
                q_diag=None, q_R=None, q_D=None, p_rowptr=None, p_colind=None, p_val=None)
    if box:
        xl = np.full(N, -np.inf)
        xh = np.full(N, np.inf)
        if x_lo is not None:
            xl[:n] = x_lo
        if x_hi is not None:
            xh[:n] = x_hi
        inst["x_lo"], inst["x_hi"] = xl, xh
    if q0_diag is not None:
        inst["q_diag"] = np.concatenate([np.asarray(q0_diag, np.float64), np.zeros(N - n)])
    if q0_R is not None:
        R0 = np.asarray(q0_R, np.float64)
        inst["q_R"] = np.concatenate([R0, np.zeros((R0.shape[0], N - n))], axis=1)
        inst["q_D"] = np.eye(R0.shape[0]) if q0_D is None else np.asarray(q0_D, np.float64)
    if q0_P is not None:
        prp = np.asarray(q0_P[0], np.int64)
        inst["p_rowptr"] = np.concatenate([prp, np.full(N - n, prp[-1], np.int64)])
        inst["p_colind"] = np.asarray(q0_P[1], np.int64)
        inst["p_val"] = np.asarray(q0_P[2], np.float64)
    return inst, (lambda x: np.asarray(x)[:n])


def lasso_to_qp(A, b, lam, m=None, n=None, name="lasso"):
    """Lasso min ||Ax - b||^2 + lam ||x||_1 -> QP min y'y + lam 1't s.t. y = Ax - b,
    -t <= x <= t (Sec. 5.5).  A is a CSR triple (m rows, n columns).

    Variables [x (n) | y (m) | t (n)], all free.  Rows: -A x + y = -b, then x_j - t_j <= 0 and
    x_j + t_j >= 0.  Q = diag(0, 2 I, 0), c = (0, 0, lam).  Returns (instance, recover)."""
    rp, ci, v = A
    rp = np.asarray(rp, np.int64)
    m = rp.size - 1 if m is None else m
    n = int(np.asarray(ci).max()) + 1 if n is None else n
    b = np.asarray(b, np.float64)
    N = 2 * n + m
    rows = _Rows(N)
    ey = _identity(m)
    rows.add(*_hstack_rows([(rp, ci, -np.asarray(v, np.float64), 0), (ey[0], ey[1], ey[2], n)], m), -b, -b)
    ex, et = _identity(n), _identity(n, -1.0)
    rows.add(*_hstack_rows([(ex[0], ex[1], ex[2], 0), (et[0], et[1], et[2], n + m)], n), -np.inf, 0.0)
    et = _identity(n)
    rows.add(*_hstack_rows([(ex[0], ex[1], ex[2], 0), (et[0], et[1], et[2], n + m)], n), 0.0, np.inf)
    a_rp, a_ci, a_v, lo, hi = rows.csr()
    bt, bs, bd, ba = _blocks([(FREE, N)])
    q = np.zeros(N)
    q[n:n + m] = 2.0
    c = np.zeros(N)
    c[n + m:] = lam
    inst = dict(name=name, m=int(lo.size), n=int(N), a_rowptr=a_rp, a_colind=a_ci, a_val=a_v, c=c,
                b=np.zeros(lo.size), row_lo=lo, row_hi=hi, blk_type=bt, blk_start=bs, blk_dim=bd, blk_alpha=ba,
                q_diag=q, q_R=None, q_D=None, p_rowptr=None, p_colind=None, p_val=None)
    return inst, (lambda x: np.asarray(x)[:n])
