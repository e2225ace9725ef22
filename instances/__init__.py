"""Seeded synthetic conic-QP instances (inputs only; no solver arithmetic).

Both the FP64 CPU oracle and the CUDA path consume these instances; this module
computes nothing that the method computes.  Every random number comes from
Philox-4x32-10, the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC 2011), implemented here from
that published definition (10 rounds of the 4x32 Philox S-box with the two
published multipliers and Weyl key increments).

An instance is a plain dict of numpy arrays describing

    min 1/2 x'Qx + c'x   s.t.  A x = b,  x in K = K_1 x ... x K_J,

with A in CSR form (rowptr int64, colind int64, val float64), Q given in the
structured form Q = diag(q) + P + R' D R (any part may be absent), and K given
as a list of contiguous cone blocks (type, start, dim, alpha) that partition
0..n-1.  Cone types: 0 free, 1 nonnegative, 2 second-order (v, t) with t last,
3 rotated second-order (v, s, t) with ||v||^2 <= 2 s t, 4 exponential (r, s, t)
with s exp(r/s) <= t, 5 three-dimensional power (r, s, t) with
r^alpha s^(1-alpha) >= |t|.
"""
from __future__ import annotations

import numpy as np

CONE_FREE, CONE_NONNEG, CONE_SOC, CONE_RSOC, CONE_EXP, CONE_POW = 0, 1, 2, 3, 4, 5
# exponential / power blocks whose middle coordinate is fixed at one (no affine row for it)
CONE_EXP1, CONE_POW1 = 7, 8

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox-4x32-10 block function.

    ctr: uint32 array of shape (N, 4); key: uint32 array of shape (2,) or (N, 2).
    Returns uint32 array (N, 4).
    """
    c = np.array(ctr, dtype=np.uint32, copy=True).reshape(-1, 4)
    k = np.broadcast_to(np.asarray(key, dtype=np.uint32), (c.shape[0], 2)).copy()
    c0, c1, c2, c3 = (c[:, i].astype(np.uint64) for i in range(4))
    k0 = k[:, 0].astype(np.uint64)
    k1 = k[:, 1].astype(np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(_W0)) & _MASK32
            k1 = (k1 + np.uint64(_W1)) & _MASK32
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


class Stream:
    """A Philox stream keyed by (seed, stream id); counters advance sequentially."""

    def __init__(self, seed: int, stream: int = 0):
        self.key = np.array([seed & 0xFFFFFFFF, stream & 0xFFFFFFFF], dtype=np.uint32)
        self.counter = 0

    def u32(self, n: int) -> np.ndarray:
        nblk = (n + 3) // 4
        idx = np.arange(self.counter, self.counter + nblk, dtype=np.uint64)
        self.counter += nblk
        ctr = np.zeros((nblk, 4), dtype=np.uint32)
        ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
        ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
        return philox4x32_10(ctr, self.key).reshape(-1)[:n]

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Doubles in [lo, hi) with 53 random bits each (two 32-bit draws)."""
        w = self.u32(2 * n).astype(np.uint64).reshape(n, 2)
        m = ((w[:, 0] >> np.uint64(5)) << np.uint64(26)) | (w[:, 1] >> np.uint64(6))
        u = m.astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
        """Box-Muller normals."""
        h = (n + 1) // 2
        u1 = self.uniform(h)
        u2 = self.uniform(h)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])[:n]
        return mean + std * z

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers uniform in [lo, hi) (hi - lo < 2**31)."""
        span = hi - lo
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def _coo_to_csr(m, n, rows, cols, vals):
    """Sum duplicates and return CSR arrays with sorted column indices."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size:
        key = rows * n + cols
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        grp = np.cumsum(first) - 1
        vals = np.bincount(grp, weights=vals)
        rows, cols = rows[first], cols[first]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols, vals


def csr_matvec(rowptr, colind, val, x):
    """Plain CSR product used only to build right-hand sides b = A x0."""
    m = rowptr.size - 1
    prod = val * x[colind]
    out = np.zeros(m)
    nz = np.diff(rowptr)
    rows = np.repeat(np.arange(m), nz)
    np.add.at(out, rows, prod)
    return out


def blocks_from_list(blist):
    """blist: list of (type, dim, alpha) in order -> block arrays."""
    t = np.array([b[0] for b in blist], dtype=np.int32)
    d = np.array([b[1] for b in blist], dtype=np.int64)
    a = np.array([b[2] for b in blist], dtype=np.float64)
    s = np.zeros_like(d)
    if d.size:
        s[1:] = np.cumsum(d)[:-1]
    return t, s, d, a


def interior_point(stream: Stream, btype, bstart, bdim, balpha, n):
    """A point strictly inside K (used as a feasible x0 so that b = A x0)."""
    x = np.zeros(n)
    for t, s, d, al in zip(btype, bstart, bdim, balpha):
        s, d = int(s), int(d)
        if t == CONE_FREE:
            x[s:s + d] = stream.normal(d)
        elif t == CONE_NONNEG:
            x[s:s + d] = np.abs(stream.normal(d)) + 0.01
        elif t == CONE_SOC:
            v = stream.normal(d - 1)
            x[s:s + d - 1] = v
            x[s + d - 1] = np.linalg.norm(v) + abs(stream.normal(1)[0]) + 0.1
        elif t == CONE_RSOC:
            v = stream.normal(d - 2)
            sv = abs(stream.normal(1)[0]) + 0.5
            x[s:s + d - 2] = v
            x[s + d - 2] = sv
            x[s + d - 1] = v @ v / (2 * sv) + abs(stream.normal(1)[0]) + 0.1
        elif t == CONE_EXP:
            r = stream.normal(1)[0]
            sv = abs(stream.normal(1)[0]) + 0.5
            x[s:s + 3] = [r, sv, sv * np.exp(r / sv) + abs(stream.normal(1)[0]) + 0.1]
        elif t == CONE_POW:
            r = abs(stream.normal(1)[0]) + 0.5
            sv = abs(stream.normal(1)[0]) + 0.5
            bound = r ** al * sv ** (1 - al)
            x[s:s + 3] = [r, sv, 0.5 * bound * (2 * stream.uniform(1)[0] - 1)]
    return x


def make_instance(name, m, n, a_rowptr, a_colind, a_val, c, b, btype, bstart, bdim, balpha,
                  q_diag=None, p_csr=None, q_R=None, q_D=None, **extra):
    inst = dict(name=name, m=int(m), n=int(n),
                a_rowptr=np.ascontiguousarray(a_rowptr, dtype=np.int64),
                a_colind=np.ascontiguousarray(a_colind, dtype=np.int64),
                a_val=np.ascontiguousarray(a_val, dtype=np.float64),
                c=np.ascontiguousarray(c, dtype=np.float64),
                b=np.ascontiguousarray(b, dtype=np.float64),
                blk_type=np.ascontiguousarray(btype, dtype=np.int32),
                blk_start=np.ascontiguousarray(bstart, dtype=np.int64),
                blk_dim=np.ascontiguousarray(bdim, dtype=np.int64),
                blk_alpha=np.ascontiguousarray(balpha, dtype=np.float64),
                q_diag=None if q_diag is None else np.ascontiguousarray(q_diag, dtype=np.float64),
                p_rowptr=None, p_colind=None, p_val=None,
                q_R=None if q_R is None else np.ascontiguousarray(q_R, dtype=np.float64),
                q_D=None if q_D is None else np.ascontiguousarray(q_D, dtype=np.float64))
    if p_csr is not None:
        inst["p_rowptr"] = np.ascontiguousarray(p_csr[0], dtype=np.int64)
        inst["p_colind"] = np.ascontiguousarray(p_csr[1], dtype=np.int64)
        inst["p_val"] = np.ascontiguousarray(p_csr[2], dtype=np.float64)
    inst.update(extra)
    return inst


def _random_sparse(stream, m, n, density):
    """Bernoulli(density) pattern with N(0,1) values, sampled column by column."""
    mask = stream.uniform(m * n) < density
    idx = np.nonzero(mask)[0]
    rows, cols = idx // n, idx % n
    vals = stream.normal(idx.size)
    return rows, cols, vals


# ---------------------------------------------------------------------------
# the five benchmark configurations (seed 1000 + config number)
# ---------------------------------------------------------------------------

def sparse_qp_nonneg(n=1000, m=500, a_density=0.01, m_rows=200, m_density=0.02, seed=1001):
    """Config 1: plain sparse QP over the nonnegative orthant.

    A (m x n) 1% dense N(0,1); Q = M'M + 1e-2 I with M (m_rows x n) 2% dense
    N(0,1), passed as one sparse symmetric P; c ~ N(0,1); b = A x0 with
    x0 = |N(0,1)|.
    """
    st = Stream(seed, 0)
    ar, ac, av = _random_sparse(st, m, n, a_density)
    a_rowptr, a_colind, a_val = _coo_to_csr(m, n, ar, ac, av)
    mr, mc, mv = _random_sparse(st, m_rows, n, m_density)
    Md = np.zeros((m_rows, n))
    Md[mr, mc] = mv
    Qd = Md.T @ Md + 1e-2 * np.eye(n)
    pr, pc = np.nonzero(Qd)
    p_csr = _coo_to_csr(n, n, pr, pc, Qd[pr, pc])
    c = st.normal(n)
    x0 = np.abs(st.normal(n))
    b = csr_matvec(a_rowptr, a_colind, a_val, x0)
    btype, bstart, bdim, balpha = blocks_from_list([(CONE_NONNEG, n, 0.0)])
    return make_instance("sparse_qp_nonneg_n%d_m%d" % (n, m), m, n, a_rowptr, a_colind, a_val, c, b,
                         btype, bstart, bdim, balpha, p_csr=p_csr, x_feasible=x0)


def socp_mix(n=200_000, n_nonneg=100_000, n_soc=2000, soc_dim=(10, 50), n_rsoc=500, rsoc_dim=(3, 20),
             m=100_000, nnz_per_col=10, rank=20, seed=1002):
    """Config 2: SOCP/QCQP mix with diagonal-plus-low-rank Q.

    Blocks in order: n_nonneg nonnegative coordinates, n_soc SOCs of dimension
    U[soc_dim], n_rsoc rotated SOCs of dimension U[rsoc_dim], then free
    coordinates up to n.  A has about nnz_per_col N(0,1) entries per column and
    every row at least one entry; Q = diag(lognormal(0,1)) + R'R with R (rank x n)
    N(0, 1/n); c ~ N(0,1); b = A x0 with x0 strictly inside K.
    """
    st = Stream(seed, 0)
    blist = [(CONE_NONNEG, n_nonneg, 0.0)]
    sd = st.integers(n_soc, soc_dim[0], soc_dim[1] + 1)
    rd = st.integers(n_rsoc, rsoc_dim[0], rsoc_dim[1] + 1)
    blist += [(CONE_SOC, int(d), 0.0) for d in sd]
    blist += [(CONE_RSOC, int(d), 0.0) for d in rd]
    used = sum(b[1] for b in blist)
    if used > n:
        raise ValueError("cone blocks exceed n")
    if n - used > 0:
        blist.append((CONE_FREE, n - used, 0.0))
    btype, bstart, bdim, balpha = blocks_from_list(blist)
    cols = np.repeat(np.arange(n, dtype=np.int64), nnz_per_col)
    rows = st.integers(cols.size, 0, m)
    vals = st.normal(cols.size)
    present = np.zeros(m, dtype=bool)
    present[rows] = True
    empty = np.nonzero(~present)[0]
    if empty.size:
        rows = np.concatenate([rows, empty])
        cols = np.concatenate([cols, st.integers(empty.size, 0, n)])
        vals = np.concatenate([vals, st.normal(empty.size)])
    a_rowptr, a_colind, a_val = _coo_to_csr(m, n, rows, cols, vals)
    q_diag = np.exp(st.normal(n))
    q_R = st.normal(rank * n, 0.0, 1.0 / np.sqrt(n)).reshape(rank, n)
    q_D = np.eye(rank)
    c = st.normal(n)
    x0 = interior_point(st, btype, bstart, bdim, balpha, n)
    b = csr_matvec(a_rowptr, a_colind, a_val, x0)
    return make_instance("socp_mix_n%d_m%d" % (n, m), m, n, a_rowptr, a_colind, a_val, c, b,
                         btype, bstart, bdim, balpha, q_diag=q_diag, q_R=q_R, q_D=q_D, x_feasible=x0)


def fisher_market(n_buyers=10_000, n_goods=1000, density=0.05, seed=1003, pow_fraction=0.5, fixed_middle=True):
    """Config 3: quasilinear Fisher market with exponential and power cones.

    Variables, in order: allocations x_ij on the valuation graph E (nonneg),
    retained money delta_i (nonneg), then one 3-D block per buyer:
    exponential (z_i, s_i, t_i) with s_i exp(z_i/s_i) <= t_i, or power
    (t_i, s_i, z_i) with t_i^a s_i^(1-a) >= |z_i|, where s_i = 1.  Rows: supply
    sum_i x_ij = 1 (one per good) and utility t_i - sum_j u_ij x_ij - delta_i = 0
    (one per buyer).  With fixed_middle (the form of eq. fisher-conic: e + 4n
    stored coordinates, m + n equations) s_i = 1 is part of the block type
    (CONE_EXP1 / CONE_POW1); otherwise the blocks are cones and one row s_i = 1
    per buyer is added (m + 2n rows).  Objective sum_i (delta_i - w_i z_i),
    Q = 0.  Valuations lognormal(0,1) at the given density, budgets
    w_i ~ U[0.5, 2], supplies 1, alpha ~ U[0.2, 0.8].
    """
    st = Stream(seed, 0)
    nb, ng = n_buyers, n_goods
    mask = st.uniform(nb * ng) < density
    idx = np.nonzero(mask)[0]
    bi, gj = idx // ng, idx % ng
    # every good needs at least one buyer and every buyer at least one good
    missing_g = np.setdiff1d(np.arange(ng), gj)
    if missing_g.size:
        bi = np.concatenate([bi, st.integers(missing_g.size, 0, nb)])
        gj = np.concatenate([gj, missing_g])
    missing_b = np.setdiff1d(np.arange(nb), bi)
    if missing_b.size:
        bi = np.concatenate([bi, missing_b])
        gj = np.concatenate([gj, st.integers(missing_b.size, 0, ng)])
    order = np.lexsort((gj, bi))
    bi, gj = bi[order], gj[order]
    e = bi.size
    u = np.exp(st.normal(e))
    w = st.uniform(nb, 0.5, 2.0)
    is_pow = st.uniform(nb) < pow_fraction
    alpha = st.uniform(nb, 0.2, 0.8)
    n = e + nb + 3 * nb
    off_delta = e
    off_cone = e + nb
    blist = [(CONE_NONNEG, e + nb, 0.0)]
    t_exp, t_pow = (CONE_EXP1, CONE_POW1) if fixed_middle else (CONE_EXP, CONE_POW)
    for i in range(nb):
        blist.append((t_pow, 3, float(alpha[i])) if is_pow[i] else (t_exp, 3, 0.0))
    btype, bstart, bdim, balpha = blocks_from_list(blist)
    # coordinate of z_i, s_i, t_i inside block i
    zc = np.where(is_pow, 2, 0)
    tc = np.where(is_pow, 0, 2)
    z_idx = off_cone + 3 * np.arange(nb) + zc
    s_idx = off_cone + 3 * np.arange(nb) + 1
    t_idx = off_cone + 3 * np.arange(nb) + tc
    rows = [gj, ng + bi, ng + np.arange(nb), ng + np.arange(nb)]
    cols = [np.arange(e), np.arange(e), t_idx, off_delta + np.arange(nb)]
    vals = [np.ones(e), -u, np.ones(nb), -np.ones(nb)]
    b = [np.ones(ng), np.zeros(nb)]
    if not fixed_middle:
        rows.append(ng + nb + np.arange(nb))
        cols.append(s_idx)
        vals.append(np.ones(nb))
        b.append(np.ones(nb))
    m = ng + nb * (1 if fixed_middle else 2)
    a_rowptr, a_colind, a_val = _coo_to_csr(m, n, np.concatenate(rows), np.concatenate(cols),
                                            np.concatenate(vals))
    b = np.concatenate(b)
    c = np.zeros(n)
    c[off_delta:off_delta + nb] = 1.0
    c[z_idx] = -w
    return make_instance("fisher_b%d_g%d" % (nb, ng), m, n, a_rowptr, a_colind, a_val, c, b,
                         btype, bstart, bdim, balpha, q_diag=np.zeros(n),
                         fisher=dict(n_buyers=nb, n_goods=ng, edges=e, buyer=bi, good=gj, u=u, w=w,
                                     is_pow=is_pow, alpha=alpha, z_idx=z_idx, t_idx=t_idx, s_idx=s_idx,
                                     fixed_middle=fixed_middle))



def portfolio_instance(n, k, stream):
    """One long-only factor-model portfolio QP (config 4 building block).

    Variables, in order: weights x (n, nonnegative), then one second-order cone
    block (w_F (k), w_D (n), t) with t last.  Rows: 1'x = 1; F'x - w_F = 0 (k);
    D^(1/2) x - w_D = 0 (n); t = sigma_bar.  Objective 1/2 x'(F F' + D) x - mu'x,
    given as Q = diag(D on x) + R' R with R = F' on the x coordinates.  F ~ N(0,
    0.1^2) (n x k), D ~ U[0.01, 0.1], mu ~ N(0.05, 0.02^2); sigma_bar is the risk
    ||(F'x_eq, D^(1/2) x_eq)|| of the equal-weight portfolio, which is therefore
    feasible.  Returns a dict of per-instance arrays (local indices).
    """
    F = stream.normal(n * k, 0.0, 0.1).reshape(n, k)
    Dg = stream.uniform(n, 0.01, 0.1)
    mu = stream.normal(n, 0.05, 0.02)
    xeq = np.full(n, 1.0 / n)
    sigma_bar = float(np.sqrt(np.sum((F.T @ xeq) ** 2) + np.sum(Dg * xeq ** 2)))
    nv = 2 * n + k + 1
    m = n + k + 2
    # CSR rows built directly: budget, k factor rows, n idiosyncratic rows, risk bound
    lens = np.concatenate([[n], np.full(k, n + 1), np.full(n, 2), [1]]).astype(np.int64)
    rowptr = np.zeros(m + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    xs = np.arange(n, dtype=np.int64)
    fac_cols = np.concatenate([np.concatenate([xs, [n + l]]) for l in range(k)]) if k else np.zeros(0, np.int64)
    fac_vals = np.concatenate([np.concatenate([F[:, l], [-1.0]]) for l in range(k)]) if k else np.zeros(0)
    idio_cols = np.stack([xs, n + k + xs], axis=1).ravel()
    idio_vals = np.stack([np.sqrt(Dg), -np.ones(n)], axis=1).ravel()
    colind = np.concatenate([xs, fac_cols, idio_cols, [2 * n + k]]).astype(np.int64)
    val = np.concatenate([np.ones(n), fac_vals, idio_vals, [1.0]])
    b = np.concatenate([[1.0], np.zeros(k + n), [sigma_bar]])
    c = np.concatenate([-mu, np.zeros(k + n + 1)])
    q = np.concatenate([Dg, np.zeros(k + n + 1)])
    return dict(n=nv, m=m, n_assets=n, k=k, rowptr=rowptr, colind=colind, val=val, b=b, c=c, q=q, F=F,
                blocks=[(CONE_NONNEG, n, 0.0), (CONE_SOC, k + n + 1, 0.0)])


def portfolio_batch(count=4096, n_range=(50, 2000), k_range=(10, 50), seed=1004):
    """Config 4: a batch of uneven portfolio QPs as one block-diagonal problem.

    Instance i has n_i ~ U[n_range] assets and k_i ~ U[k_range] factors (see
    portfolio_instance).  The instances are concatenated: coordinates and rows
    of instance i occupy [x_off[i], x_off[i+1]) and [row_off[i], row_off[i+1]);
    the low-rank factor R is max_i k_i rows by n columns, instance i filling
    rows 0..k_i-1 of its own x columns, with D = I.
    """
    st = Stream(seed, 0)
    ns = st.integers(count, n_range[0], n_range[1] + 1)
    ks = st.integers(count, k_range[0], k_range[1] + 1)
    parts = [portfolio_instance(int(ns[i]), int(ks[i]), Stream(seed, 1 + i)) for i in range(count)]
    x_off = np.zeros(count + 1, np.int64)
    row_off = np.zeros(count + 1, np.int64)
    x_off[1:] = np.cumsum([p["n"] for p in parts])
    row_off[1:] = np.cumsum([p["m"] for p in parts])
    n, m = int(x_off[-1]), int(row_off[-1])
    nnz_off = np.zeros(count + 1, np.int64)
    nnz_off[1:] = np.cumsum([p["rowptr"][-1] for p in parts])
    a_rowptr = np.zeros(m + 1, np.int64)
    a_colind = np.empty(int(nnz_off[-1]), np.int64)
    a_val = np.empty(int(nnz_off[-1]))
    c = np.empty(n)
    b = np.empty(m)
    q = np.empty(n)
    K = int(ks.max()) if count else 0
    R = np.zeros((K, n))
    blist = []
    for i, p in enumerate(parts):
        r0, x0, z0 = row_off[i], x_off[i], nnz_off[i]
        a_rowptr[r0 + 1:row_off[i + 1] + 1] = p["rowptr"][1:] + z0
        a_colind[z0:nnz_off[i + 1]] = p["colind"] + x0
        a_val[z0:nnz_off[i + 1]] = p["val"]
        c[x0:x_off[i + 1]] = p["c"]
        b[r0:row_off[i + 1]] = p["b"]
        q[x0:x_off[i + 1]] = p["q"]
        R[:p["k"], x0:x0 + p["n_assets"]] = p["F"].T
        blist.extend(p["blocks"])
    btype, bstart, bdim, balpha = blocks_from_list(blist)
    inst = make_instance("portfolio_batch_%d" % count, m, n, a_rowptr, a_colind, a_val, c, b, btype, bstart,
                         bdim, balpha, q_diag=q, q_R=R, q_D=np.eye(K))
    inst.update(batch_count=count, x_off=x_off, row_off=row_off, n_assets=ns.astype(np.int64),
                n_factors=ks.astype(np.int64))
    return inst


def batch_member(inst, i):
    """Instance i of a block-diagonal batch as a stand-alone instance dict."""
    x0, x1 = int(inst["x_off"][i]), int(inst["x_off"][i + 1])
    r0, r1 = int(inst["row_off"][i]), int(inst["row_off"][i + 1])
    rp = inst["a_rowptr"]
    z0, z1 = int(rp[r0]), int(rp[r1])
    sel = (inst["blk_start"] >= x0) & (inst["blk_start"] < x1)
    R = None if inst.get("q_R") is None else inst["q_R"][:, x0:x1]
    return make_instance("%s[%d]" % (inst["name"], i), r1 - r0, x1 - x0, rp[r0:r1 + 1] - z0,
                         inst["a_colind"][z0:z1] - x0, inst["a_val"][z0:z1], inst["c"][x0:x1], inst["b"][r0:r1],
                         inst["blk_type"][sel], inst["blk_start"][sel] - x0, inst["blk_dim"][sel],
                         inst["blk_alpha"][sel],
                         q_diag=None if inst.get("q_diag") is None else inst["q_diag"][x0:x1],
                         q_R=R, q_D=inst.get("q_D"))


# ---------------------------------------------------------------------------
# index-addressed draws (random access, for instances generated on the device)
# ---------------------------------------------------------------------------

def philox_at(seed, stream, idx):
    """Philox-4x32-10 block of counter (idx_lo, idx_hi, 0, 0) under key (seed, stream)."""
    idx = np.asarray(idx, dtype=np.uint64).reshape(-1)
    ctr = np.zeros((idx.size, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, stream & 0xFFFFFFFF], dtype=np.uint32)
    return philox4x32_10(ctr, key)


def _u53(w_hi, w_lo):
    m = ((w_hi.astype(np.uint64) >> np.uint64(5)) << np.uint64(26)) | (w_lo.astype(np.uint64) >> np.uint64(6))
    return m.astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_at(seed, stream, idx):
    """U[0,1) with 53 bits from words 0 and 1 of the block of index idx."""
    w = philox_at(seed, stream, idx)
    return _u53(w[:, 0], w[:, 1])


def normal_at(seed, stream, idx):
    """N(0,1) by Box-Muller from the block of index idx (words 0,1 -> u1, words 2,3 -> u2)."""
    w = philox_at(seed, stream, idx)
    u1 = _u53(w[:, 0], w[:, 1])
    u2 = _u53(w[:, 2], w[:, 3])
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


LARGE_NNZ_PER_ROW = 20


def large_qp(n=200_000_000, m=50_000_000, seed=1005):
    """Config 5 (any size): large sparse QP over the nonnegative orthant.

    A (m x n): row r has 20 entries, slot e drawing column floor(U * n) from stream 1
    and value N(0,1) from stream 2 at index 20 r + e; a row's entries are sorted by
    column (ties by slot) and a repeated column keeps the sum of its values in its
    first entry and an explicit 0 in the others, so every row keeps 20 stored entries
    (about 5 per column on average).  Q = diag(q) + S: q_j ~ U[0,1] (stream 5) and S
    the Laplacian of a perfect matching j <-> j + d (j even, indices mod n, d odd from
    stream 7) with pair weight |N(0,1)| (stream 6, at the even endpoint), given as P
    with rows {j: w, partner: -w} in column order.  c_j ~ N(0,1) (stream 3),
    b = A x0 with x0_j = |N(0,1)| (stream 4), summed in stored order.  n must be even.
    Generated identically by instances.gpu.large_qp_device on the GPU.
    """
    assert n % 2 == 0
    k = LARGE_NNZ_PER_ROW
    idx = np.arange(m * k, dtype=np.uint64)
    cols = np.minimum((uniform_at(seed, 1, idx) * n).astype(np.int64), n - 1).reshape(m, k)
    vals = normal_at(seed, 2, idx).reshape(m, k)
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    for e in range(1, k):                 # repeated columns: running sum into the first entry
        dup = cols[:, e] == cols[:, e - 1]
        if dup.any():
            r = np.nonzero(dup)[0]
            first = e - 1
            while True:
                back = (first > 0) & (cols[r, np.maximum(first - 1, 0)] == cols[r, e])
                if not np.any(back):
                    break
                first = np.where(back, first - 1, first)
            vals[r, first] += vals[r, e]
            vals[r, e] = 0.0
    a_rowptr = np.arange(0, m * k + 1, k, dtype=np.int64)
    x0 = np.abs(normal_at(seed, 4, np.arange(n, dtype=np.uint64)))
    b = np.zeros(m)
    for e in range(k):
        b += vals[:, e] * x0[cols[:, e]]
    c = normal_at(seed, 3, np.arange(n, dtype=np.uint64))
    q = uniform_at(seed, 5, np.arange(n, dtype=np.uint64))
    d = 2 * int(uniform_at(seed, 7, np.zeros(1, dtype=np.uint64))[0] * (n // 2)) + 1
    j = np.arange(n, dtype=np.int64)
    even = (j % 2) == 0
    partner = np.where(even, (j + d) % n, (j - d) % n)
    anchor = np.where(even, j, partner)
    w = np.abs(normal_at(seed, 6, anchor.astype(np.uint64)))
    lo_first = j < partner
    p_colind = np.stack([np.where(lo_first, j, partner), np.where(lo_first, partner, j)], axis=1).ravel()
    p_val = np.stack([np.where(lo_first, w, -w), np.where(lo_first, -w, w)], axis=1).ravel()
    p_rowptr = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    btype, bstart, bdim, balpha = blocks_from_list([(CONE_NONNEG, n, 0.0)])
    return make_instance("large_qp_n%d_m%d" % (n, m), m, n, a_rowptr, cols.ravel(), vals.ravel(), c, b,
                         btype, bstart, bdim, balpha, q_diag=q, p_csr=(p_rowptr, p_colind, p_val), x_feasible=x0)

# ---------------------------------------------------------------------------
# original-form problems for the modeling front-ends (no reformulation here)
# ---------------------------------------------------------------------------

def _rows_uniform(stream, m, n, per_row):
    """CSR with per_row[i] uniform columns in row i (repeats summed) and N(0,1) values."""
    per_row = np.asarray(per_row, dtype=np.int64)
    tot = int(per_row.sum())
    rows = np.repeat(np.arange(m, dtype=np.int64), per_row)
    cols = stream.integers(tot, 0, n)
    vals = stream.normal(tot)
    return _coo_to_csr(m, n, rows, cols, vals)


def lasso_problem(m=677_399, n=47_236, density=1.55e-3, seed=1006, support=0.1, noise=0.1):
    """Synthetic Lasso data min ||Ax - b||^2 + lam ||x||_1 with the shape and density of the
    rcv1_test instance of the paper's Lasso table (its values are not used: A has a
    Poisson(n density) number of uniform columns per row with N(0,1)/sqrt(row count)
    values, b = A x_true + noise with a support-fraction sparse x_true).  lam is the
    paper's 0.01 ||A'b||_inf."""
    st = Stream(seed, 0)
    lam_row = n * density
    # Poisson counts by inversion of uniforms is slow for large means: use the normal
    # approximation, rounded and clipped to >= 1 (every sample has a feature)
    cnt = np.maximum(1, np.rint(lam_row + np.sqrt(lam_row) * st.normal(m))).astype(np.int64)
    rp, ci, v = _rows_uniform(st, m, n, cnt)
    v = v / np.sqrt(np.repeat(np.diff(rp), np.diff(rp)).astype(np.float64))
    xt = np.zeros(n)
    k = max(1, int(support * n))
    idx = st.integers(k, 0, n)
    xt[idx] = st.normal(k)
    b = csr_matvec(rp, ci, v, xt) + noise * st.normal(m)
    aty = np.zeros(n)
    np.add.at(aty, ci, v * np.repeat(b, np.diff(rp)))
    lam = 0.01 * float(np.abs(aty).max())
    return dict(m=m, n=n, a_rowptr=rp, a_colind=ci, a_val=v, b=b, lam=lam, x_true=xt)


def qcqp_problem(n=2000, m_lin=500, p=5, k=20, k0=10, lin_per_row=10, quad_per_row=20, seed=1007, box=1.0,
                 c_nnz=None):
    """Synthetic convex QCQP in the form of eq. qcqp-benchmark-form:
        min 1/2 x'Q0 x + c0'x  s.t.  lo <= A x <= hi,  -box <= x <= box,
                                     1/2 ||R_i x||^2 + c_i'x <= d_i  (Q_i = R_i'R_i), i = 1..p
    Q0 = diag(q0) + R0'R0 (q0 ~ U[0.1, 1], R0 k0 x n N(0, 1/n)); A has lin_per_row
    N(0,1) entries per row; R_i has k rows with quad_per_row N(0,1) entries each; c_i
    ~ N(0, 0.1^2) (dense, or c_nnz uniform positions when given).  x0 ~ U(-box/2, box/2) is strictly feasible: the rows get bounds
    A x0 -/+ U[0.1, 1] (a third one-sided), and d_i = value at x0 + U[0.05, 0.5].
    c0 ~ N(0,1) pulls the optimum onto the constraints."""
    st = Stream(seed, 0)
    x0 = st.uniform(n, -0.5 * box, 0.5 * box)
    q0 = st.uniform(n, 0.1, 1.0)
    R0 = st.normal(k0 * n, 0.0, 1.0 / np.sqrt(n)).reshape(k0, n)
    c0 = st.normal(n)
    arp, aci, av = _rows_uniform(st, m_lin, n, np.full(m_lin, lin_per_row))
    ax0 = csr_matvec(arp, aci, av, x0)
    lo = ax0 - st.uniform(m_lin, 0.1, 1.0)
    hi = ax0 + st.uniform(m_lin, 0.1, 1.0)
    third = m_lin // 3
    lo[:third] = -np.inf
    quad = []
    for _ in range(p):
        rrp, rci, rv = _rows_uniform(st, k, n, np.full(k, quad_per_row))
        if c_nnz is None:
            ci = st.normal(n, 0.0, 0.1)
        else:
            ci = np.zeros(n)
            ci[st.integers(c_nnz, 0, n)] = st.normal(c_nnz, 0.0, 0.1)
        rx = csr_matvec(rrp, rci, rv, x0)
        d = 0.5 * float(rx @ rx) + float(ci @ x0) + float(st.uniform(1, 0.05, 0.5)[0])
        quad.append(dict(R=(rrp, rci, rv), k=k, c=ci, d=d))
    return dict(n=n, c0=c0, q0_diag=q0, q0_R=R0, A=(arp, aci, av), m_lin=m_lin, row_lo=lo, row_hi=hi,
                x_lo=np.full(n, -box), x_hi=np.full(n, box), quad=quad, x_feasible=x0)


CONFIGS = {
    1: lambda: sparse_qp_nonneg(),
    2: lambda: socp_mix(),
    3: lambda: fisher_market(),
    4: lambda: portfolio_batch(),
}
# config 5 (n = 2e8, m = 5e7, 1e9 nonzeros) is generated on the device: instances.gpu.large_qp_device


def round_bf16(a) -> np.ndarray:
    """Values rounded to FP32, then to BF16 (round to nearest, ties to even, at each step),
    returned as FP64: the matrix values a solve with BF16 matrix storage works with."""
    f = np.ascontiguousarray(a, dtype=np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a) -> np.ndarray:
    """The BF16 bit patterns (uint16) of round_bf16(a)."""
    r = round_bf16(a).astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def with_bf16_matrices(inst: dict, p: bool = True) -> dict:
    """A copy of the instance with the values of A (and, if p, of the sparse part P of Q)
    rounded as round_bf16 rounds them."""
    out = dict(inst)
    out["a_val"] = round_bf16(inst["a_val"])
    if p and inst.get("p_val") is not None:
        out["p_val"] = round_bf16(inst["p_val"])
    return out


def small_config(k: int):
    """Scaled-down copies with the same structure, for oracle-speed parity tests."""
    if k == 1:
        return sparse_qp_nonneg(n=200, m=100, seed=2001)
    if k == 2:
        return socp_mix(n=3000, n_nonneg=1500, n_soc=30, n_rsoc=10, m=1500, seed=2002)
    if k == 3:
        return fisher_market(n_buyers=200, n_goods=40, density=0.1, seed=2003)
    if k == 4:
        return portfolio_batch(count=12, n_range=(20, 60), k_range=(3, 8), seed=2004)
    if k == 5:
        return large_qp(n=20_000, m=5_000, seed=2005)
    raise KeyError(k)
