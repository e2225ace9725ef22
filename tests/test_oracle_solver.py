"""Pins for the oracle's linear algebra, KKT measure, rescaling, prox and PDHG loop.

Everything is compared with facts fixed independently of the oracle code: dense
numpy products, numpy.linalg, closed-form optima of small QPs, the resolvent
identity and Fejer monotonicity of the exact PDHG step (Sec. 2, Lemma
"one-step-energy" and eq. pdhg-residual-kkt), and the reflected-Halpern residual
bound (eq. rh-residual-decay).
"""
import math
import os

import numpy as np
import pytest

import _cones as G
import instances as I


# --------------------------------------------------------------------------- helpers

def dense(rowptr, colind, val, n):
    m = rowptr.size - 1
    A = np.zeros((m, n))
    for i in range(m):
        for k in range(rowptr[i], rowptr[i + 1]):
            A[i, colind[k]] += val[k]
    return A


def csr(A):
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(A.shape[0] + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int64), A[rows, cols].astype(float)


def qp(A, c, b, blocks, Qdiag=None, P=None, R=None, D=None):
    """Build an instance dict from dense data; blocks = list of (type, dim, alpha)."""
    m, n = A.shape
    rp, ci, v = csr(A)
    bt, bs, bd, ba = I.blocks_from_list(blocks)
    pc = None if P is None else csr(P)
    return I.make_instance("t", m, n, rp, ci, v, c, b, bt, bs, bd, ba, q_diag=Qdiag, p_csr=pc, q_R=R, q_D=D)


def dense_q(inst):
    n = inst["n"]
    Q = np.zeros((n, n))
    if inst["q_diag"] is not None:
        Q += np.diag(inst["q_diag"])
    if inst["p_rowptr"] is not None:
        Q += dense(inst["p_rowptr"], inst["p_colind"], inst["p_val"], n)
    if inst["q_R"] is not None:
        Q += inst["q_R"].T @ inst["q_D"] @ inst["q_R"]
    return Q


def simplex_qp(rng, n=8):
    """min 1/2||x||^2 + c'x s.t. 1'x = 1, x >= 0: x* = projection of -c onto the simplex."""
    c = rng.normal(size=n)
    z = -c
    srt = np.sort(z)[::-1]
    css = np.cumsum(srt) - 1.0
    k = np.nonzero(srt - css / np.arange(1, n + 1) > 0)[0][-1]
    theta = css[k] / (k + 1)
    xs = np.maximum(z - theta, 0)
    ys = np.array([-theta])          # from x_i + c_i - y = 0 on the support
    inst = qp(np.ones((1, n)), c, np.array([1.0]), [(G.NONNEG, n, 0)], Qdiag=np.ones(n))
    return inst, xs, ys


# --------------------------------------------------------------------------- products

def test_spmv_exact_on_integers(orc, rng):
    A = rng.integers(-5, 6, size=(40, 30)) * (rng.uniform(size=(40, 30)) < 0.3)
    x = rng.integers(-9, 10, size=30).astype(float)
    y = rng.integers(-9, 10, size=40).astype(float)
    rp, ci, v = csr(A.astype(float))
    assert np.array_equal(orc.spmv(rp, ci, v, x), A @ x)
    assert np.array_equal(orc.spmv_t(rp, ci, v, y, 30), A.T @ y)


def test_spmv_random_within_rounding_bound(orc, rng):
    A = rng.normal(size=(60, 80)) * (rng.uniform(size=(60, 80)) < 0.2)
    x = rng.normal(size=80)
    rp, ci, v = csr(A)
    y = orc.spmv(rp, ci, v, x)
    for i in range(60):
        exact = math.fsum(A[i] * x)
        k = rp[i + 1] - rp[i]
        bound = 1.01 * k * np.finfo(float).eps * float(np.abs(A[i]) @ np.abs(x))
        assert abs(y[i] - exact) <= bound + 1e-300


def test_q_apply_against_dense(orc, rng):
    n, k = 30, 4
    P = rng.normal(size=(n, n)) * (rng.uniform(size=(n, n)) < 0.1)
    P = P + P.T
    R = rng.normal(size=(k, n))
    D = rng.normal(size=(k, k))
    D = D @ D.T
    inst = qp(np.ones((1, n)), np.zeros(n), np.ones(1), [(G.FREE, n, 0)], Qdiag=rng.uniform(size=n), P=P, R=R, D=D)
    x = rng.normal(size=n)
    assert np.allclose(orc.q_apply(inst, x), dense_q(inst) @ x, rtol=1e-13, atol=1e-12)


def test_norm_estimate(orc, rng):
    for shape in [(30, 50), (80, 40)]:
        A = rng.normal(size=shape) * (rng.uniform(size=shape) < 0.3)
        rp, ci, v = csr(A)
        s, it = orc.norm_est(rp, ci, v, shape[1], iters=2000, tol=1e-12)
        assert abs(s - np.linalg.norm(A, 2)) <= 1e-6 * np.linalg.norm(A, 2)


# --------------------------------------------------------------------------- KKT

def test_kkt_zero_at_closed_form_optimum(orc, rng):
    inst, xs, ys = simplex_qp(rng)
    rep = orc.kkt(inst, xs, ys)
    assert rep["rel_kkt"] < 1e-14
    assert abs(rep["pobj"] - (0.5 * xs @ xs + inst["c"] @ xs)) < 1e-14


def test_kkt_components_by_hand(orc, rng):
    # nonneg + SOC + free blocks; residuals recomputed in numpy with closed-form projections
    n, m = 9, 4
    A = rng.normal(size=(m, n))
    blocks = [(G.NONNEG, 3, 0), (G.SOC, 4, 0), (G.FREE, 2, 0)]
    Qd = rng.uniform(size=n)
    inst = qp(A, rng.normal(size=n), rng.normal(size=m), blocks, Qdiag=Qd)
    x, y = rng.normal(size=n), rng.normal(size=m)
    rep = orc.kkt(inst, x, y)
    s = Qd * x + inst["c"] - A.T @ y
    ms = -s
    proj = np.concatenate([np.maximum(ms[:3], 0), orc.proj_block(G.SOC, ms[3:7]), ms[7:]])
    v, t = ms[3:6], ms[6]
    a = np.linalg.norm(v)
    soc = ms[3:7] if a <= t else (np.zeros(4) if a <= -t else np.r_[(a + t) / (2 * a) * v, (a + t) / 2])
    assert np.allclose(proj[3:7], soc)
    pobj = 0.5 * x @ (Qd * x) + inst["c"] @ x
    dobj = inst["b"] @ y - 0.5 * x @ (Qd * x)
    assert np.isclose(rep["eps_p"], np.linalg.norm(A @ x - inst["b"]) / (1 + np.linalg.norm(inst["b"])))
    assert np.isclose(rep["eps_d"], np.linalg.norm(proj) / (1 + np.linalg.norm(inst["c"])))
    assert np.isclose(rep["eps_g"], abs(pobj - dobj) / (1 + abs(pobj) + abs(dobj)))


# --------------------------------------------------------------------------- rescaling

def test_rescale_consistency_and_cone_blocks(orc):
    inst = I.small_config(2)
    sc = orc.rescale(inst)
    rp, ci, av = inst["a_rowptr"], inst["a_colind"], inst["a_val"]
    rows = np.repeat(np.arange(inst["m"]), np.diff(rp))
    assert np.allclose(sc["a_val"], av / (sc["row"][rows] * sc["col"][ci]), rtol=1e-13)
    assert np.allclose(sc["c"], inst["c"] / sc["col"] / sc["beta_c"], rtol=1e-13)
    assert np.allclose(sc["b"], inst["b"] / sc["row"] / sc["beta_b"], rtol=1e-13)
    assert abs(np.linalg.norm(inst["c"] / sc["col"]) + 1 - sc["beta_c"]) < 1e-10
    # cone-preserving mode: one factor per SOC / RSOC block (eq. cone-preserving-scaling)
    for t, s, d in zip(inst["blk_type"], inst["blk_start"], inst["blk_dim"]):
        if t in (G.SOC, G.RSOC):
            blk = sc["col"][s:s + d]
            assert np.all(blk == blk[0])


def test_ruiz_equilibrates(orc, rng):
    A = rng.normal(size=(50, 70)) * np.exp(rng.normal(size=(50, 1)) * 2) * (rng.uniform(size=(50, 70)) < 0.3)
    A[:, 0] += 1.0
    A[0, :] += 1.0
    inst = qp(A, rng.normal(size=70), rng.normal(size=50), [(G.NONNEG, 70, 0)])
    sc = orc.rescale(inst, ruiz_iters=30, pc_alpha=-1.0, bound_obj=0)
    As = dense(inst["a_rowptr"], inst["a_colind"], sc["a_val"], 70)
    assert np.allclose(np.abs(As).max(axis=1), 1.0, atol=1e-3)
    assert np.allclose(np.abs(As).max(axis=0), 1.0, atol=1e-3)


# --------------------------------------------------------------------------- prox

def test_prox_diag_closed_form_and_bb_agree(orc, rng):
    n = 40
    q = rng.uniform(0.1, 3.0, size=n)
    inst = qp(rng.normal(size=(3, n)), rng.normal(size=n), np.zeros(3), [(G.NONNEG, n, 0)], Qdiag=q)
    v = rng.normal(size=n)
    tau = 0.7
    p_diag, _ = orc.prox(inst, tau, v)
    assert np.allclose(p_diag, np.maximum((v - tau * inst["c"]) / (1 + tau * q), 0), atol=1e-15)
    p_bb, it = orc.prox(inst, tau, v, force_inner=1, eps_in=1e-13)
    assert np.allclose(p_bb, p_diag, atol=1e-11)
    p_eb, _ = orc.prox(inst, tau, v, force_inner=1, jacobi=0, eps_in=1e-13)
    assert np.allclose(p_eb, p_diag, atol=1e-10)


def test_prox_fixed_point_with_cones(orc, rng):
    # general Q over nonneg + SOC + RSOC + exp + pow blocks: the prox point p satisfies
    # p = Pi_K(p - t grad H(p)) for any t > 0 (projected-gradient fixed point)
    blocks = [(G.NONNEG, 4, 0), (G.SOC, 5, 0), (G.RSOC, 4, 0), (G.EXP, 3, 0), (G.POW, 3, 0.35), (G.FREE, 2, 0)]
    n = sum(b[1] for b in blocks)
    R = rng.normal(size=(3, n))
    inst = qp(rng.normal(size=(2, n)), rng.normal(size=n), np.zeros(2), blocks, Qdiag=rng.uniform(0.1, 1, n),
              R=R, D=np.eye(3))
    Q = dense_q(inst)
    tau = 0.5
    v = rng.normal(size=n) * 2
    p, it = orc.prox(inst, tau, v, eps_in=1e-13)
    grad = Q @ p + inst["c"] + (p - v) / tau
    for t in (1e-3, 1e-2):
        assert np.allclose(orc.proj_product(inst, p - t * grad), p, atol=1e-9)
    # Euclidean-BB variant reaches the same point
    p2, _ = orc.prox(inst, tau, v, eps_in=1e-13, jacobi=0)
    assert np.allclose(p, p2, atol=1e-8)


# --------------------------------------------------------------------------- one PDHG step

def _pnorm2(dx, dy, A, tau, sigma):
    return dx @ dx / tau + 2 * (A @ dx) @ dy + dy @ dy / sigma


def test_resolvent_identity(orc, rng):
    # M(z - Tz) in F_KKT(Tz) (eq. pdhg-residual-kkt): with z+ = Tz,
    #   g = (x - x+)/tau + A'(y - y+) - (Q x+ + c - A'y+)  lies in N_K(x+)  and
    #   A(x - x+) + (y - y+)/sigma = A x+ - b.
    blocks = [(G.NONNEG, 5, 0), (G.SOC, 4, 0), (G.EXP, 3, 0)]
    n, m = 12, 4
    A = rng.normal(size=(m, n))
    inst = qp(A, rng.normal(size=n), rng.normal(size=m), blocks, Qdiag=rng.uniform(0.1, 1, n),
              R=rng.normal(size=(2, n)), D=np.eye(2))
    Q = dense_q(inst)
    tau = sigma = 0.9 / np.linalg.norm(A, 2)
    x, y = rng.normal(size=n), rng.normal(size=m)
    xp, yp, _ = orc.pdhg_operator(inst, tau, sigma, x, y, eps_in=1e-13)
    g = (x - xp) / tau + A.T @ (y - yp) - (Q @ xp + inst["c"] - A.T @ yp)
    assert np.allclose(A @ (x - xp) + (y - yp) / sigma, A @ xp - inst["b"], atol=1e-11)
    # g in N_K(x+) <=> -g in K* and <g, x+> = 0 (blockwise)
    for t, s, d in zip(inst["blk_type"], inst["blk_start"], inst["blk_dim"]):
        assert G.in_dual_cone(t, -g[s:s + d], 0.0, 1e-7), (t, g[s:s + d])
        assert abs(g[s:s + d] @ xp[s:s + d]) < 1e-8


def test_fejer_monotone_and_halpern_bound(orc, rng):
    inst, xs, ys = simplex_qp(rng, n=10)
    A = np.ones((1, 10))
    tau = 0.5
    sigma = 0.9 / (tau * 10.0)        # tau sigma ||A||^2 < 1
    # plain PDHG: Fejer monotone in the P-metric (Lemma one-step-energy)
    x, y = rng.normal(size=10), rng.normal(size=1)
    prev = _pnorm2(x - xs, y - ys, A, tau, sigma)
    for _ in range(60):
        x, y, _ = orc.pdhg_operator(inst, tau, sigma, x, y, eps_in=1e-14)
        cur = _pnorm2(x - xs, y - ys, A, tau, sigma)
        assert cur <= prev * (1 + 1e-12) + 1e-20
        prev = cur
    # reflected Halpern from anchor a: R(h^k) <= ||a - z*||_M / (rho (k+1)), k >= 1 (eq. rh-residual-decay)
    for rho in (0.5, 1.0):
        ax, ay = rng.normal(size=10), rng.normal(size=1)
        hx, hy = ax.copy(), ay.copy()
        bound0 = math.sqrt(_pnorm2(ax - xs, ay - ys, A, tau, sigma))
        for k in range(0, 80):
            tx, ty, _ = orc.pdhg_operator(inst, tau, sigma, hx, hy, eps_in=1e-14)
            if k >= 1:
                res = math.sqrt(max(_pnorm2(hx - tx, hy - ty, A, tau, sigma), 0))
                assert res <= bound0 / (rho * (k + 1)) * (1 + 1e-9) + 1e-12
            c1 = (k + 1) / (k + 2)
            hx = c1 * (2 * rho * tx + (1 - 2 * rho) * hx) + ax / (k + 2)
            hy = c1 * (2 * rho * ty + (1 - 2 * rho) * hy) + ay / (k + 2)


# --------------------------------------------------------------------------- whole solves

def _check_solution(orc, inst, x, y, info, tol=1e-4):
    assert info["status"] == 0
    rep = orc.kkt(inst, x, y)
    assert rep["rel_kkt"] <= tol


def test_solve_simplex_closed_form(orc, rng):
    inst, xs, ys = simplex_qp(rng, n=25)
    x, y, info = orc.solve(inst, tol=1e-9, max_iter=200000)
    _check_solution(orc, inst, x, y, info, 1e-9)
    assert np.allclose(x, xs, atol=1e-7)
    assert np.allclose(y, ys, atol=1e-7)


def test_solve_equality_qp_dense_kkt(orc, rng):
    n, m = 20, 6
    A = rng.normal(size=(m, n))
    R = rng.normal(size=(5, n))
    Qd = rng.uniform(0.5, 2, n)
    inst = qp(A, rng.normal(size=n), rng.normal(size=m), [(G.FREE, n, 0)], Qdiag=Qd, R=R, D=np.eye(5))
    Q = dense_q(inst)
    K = np.block([[Q, -A.T], [A, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.r_[-inst["c"], inst["b"]])
    x, y, info = orc.solve(inst, tol=1e-9, max_iter=200000)
    _check_solution(orc, inst, x, y, info, 1e-9)
    assert np.allclose(x, sol[:n], atol=1e-6)
    assert np.allclose(y, sol[n:], atol=1e-6)


def test_solve_diag_water_filling(orc, rng):
    n = 30
    q = rng.uniform(0.5, 2, n)
    a = rng.uniform(0.5, 2, n)
    c = rng.normal(size=n)
    b = 3.0
    inst = qp(a[None, :], c, np.array([b]), [(G.NONNEG, n, 0)], Qdiag=q)
    lo, hi = -100.0, 100.0
    for _ in range(200):
        yy = 0.5 * (lo + hi)
        if a @ np.maximum((a * yy - c) / q, 0) < b:
            lo = yy
        else:
            hi = yy
    xs = np.maximum((a * yy - c) / q, 0)
    x, y, info = orc.solve(inst, tol=1e-10, max_iter=200000)
    _check_solution(orc, inst, x, y, info, 1e-10)
    assert np.allclose(x, xs, atol=1e-7) and abs(y[0] - yy) < 1e-6


@pytest.mark.parametrize("t,d", [(G.SOC, 6), (G.RSOC, 6), (G.EXP, 3), (G.POW, 3)])
def test_solve_projection_qp(orc, rng, t, d):
    # min 1/2||x - p||^2 over x in K (plus a dummy free coordinate fixed by z = 0): x* = Pi_K(p),
    # checked with the brute-force / closed-form projections of the test helpers
    p = rng.normal(size=d) * 2
    n = d + 1
    A = np.zeros((1, n))
    A[0, -1] = 1.0
    inst = qp(A, np.r_[-p, 0.0], np.zeros(1), [(t, d, 0.4), (G.FREE, 1, 0)], Qdiag=np.ones(n))
    x, y, info = orc.solve(inst, tol=1e-10, max_iter=200000)
    _check_solution(orc, inst, x, y, info, 1e-10)
    xs = x[:d]
    if t == G.EXP:
        ref = G.brute_exp(p, np.ones(3))
    elif t == G.POW:
        ref = G.brute_pow(p, np.ones(3), 0.4)
    elif t == G.SOC:
        ref = G.soc_closed(p)
    else:
        ref = G.rsoc_closed(p)
    assert np.sum((xs - p) ** 2) <= np.sum((ref - p) ** 2) + 1e-8
    assert np.allclose(xs, ref, atol=2e-4)


def test_averaged_variant_converges(orc, rng):
    inst, xs, ys = simplex_qp(rng, n=12)
    x, y, info = orc.solve(inst, update=1, avg_epoch=32, tol=1e-7, max_iter=400000)
    _check_solution(orc, inst, x, y, info, 1e-7)
    assert np.allclose(x, xs, atol=1e-5)


def test_solve_invariant_to_rescaling(orc):
    inst = I.small_config(1)
    x1, y1, i1 = orc.solve(inst, tol=1e-8, max_iter=400000)
    x2, y2, i2 = orc.solve(inst, tol=1e-8, max_iter=400000, ruiz_iters=0, pc_alpha=-1.0, bound_obj=0)
    assert i1["status"] == 0 and i2["status"] == 0
    assert np.allclose(x1, x2, atol=1e-5 * (1 + np.abs(x1).max()))   # Q positive definite: x* unique


@pytest.mark.parametrize("k", [1, 2, 3])
def test_small_configs_reach_tolerance(orc, k):
    inst = I.small_config(k)
    x, y, info = orc.solve(inst, tol=1e-4, max_iter=200000, hist_cap=4096)
    _check_solution(orc, inst, x, y, info, 1e-4)
    # the KKT of the returned point, recomputed from scratch in numpy (primal residual and gap)
    A = dense(inst["a_rowptr"], inst["a_colind"], inst["a_val"], inst["n"]) if inst["n"] <= 4000 else None
    if A is not None:
        ep = np.linalg.norm(A @ x - inst["b"]) / (1 + np.linalg.norm(inst["b"]))
        assert ep <= 1e-4
    # all primal blocks feasible (candidates are projections)
    for t, s, d, a in zip(inst["blk_type"], inst["blk_start"], inst["blk_dim"], inst["blk_alpha"]):
        assert G.in_cone(t, x[s:s + d], a, 1e-9)
    # restarts: KKT at the last check is far below the first (trend of the restarted scheme)
    h = info["hist"]
    assert h["kkt"][-1] < h["kkt"][0]


def _golden_splitmix():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_state0.txt")
    with open(path) as f:
        return [int(l, 16) for l in f if l.strip() and not l.startswith("#")]


def test_power_start_is_splitmix64(orc):
    # entry j of the start vector is 1/2 + (top 53 bits of SplitMix64 output j+1 from state 0) / 2^53
    vals = _golden_splitmix()
    ref = np.array([0.5 + (w >> 11) / 2.0 ** 53 for w in vals])
    assert np.array_equal(orc.power_start(len(vals)), ref)


def test_norm_estimate_symmetric_lasso_model(orc):
    # the Lasso reformulation with A = I after rescaling: its top singular vector is
    # orthogonal to the all-ones vector, which an all-ones start would never leave
    from oracle import frontends as OF
    b = np.random.default_rng(54).normal(size=12)
    inst = OF.lasso(np.eye(12), b, 0.8)
    sc = orc.rescale(inst)
    m, n = inst["m"], inst["n"]
    A = np.zeros((m, n))
    for i in range(m):
        for t in range(inst["a_rowptr"][i], inst["a_rowptr"][i + 1]):
            A[i, inst["a_colind"][t]] = sc["a_val"][t]
    top = np.linalg.svd(A, compute_uv=False)[0]
    assert abs(np.ones(n) @ np.linalg.svd(A)[2][0]) <= 1e-12 * np.sqrt(n)
    s, it = orc.norm_est(inst["a_rowptr"], inst["a_colind"], sc["a_val"], n)
    assert abs(s - top) <= 1e-5 * top


def test_tridiagonal_max_eigenvalue(orc):
    # the Lanczos step's eigenvalue search against LAPACK on random, clustered and scaled cases
    rng = np.random.default_rng(91)
    cases = [(rng.normal(size=k), rng.normal(size=k - 1)) for k in (1, 2, 3, 7, 30, 200)]
    cases += [(np.ones(20), 1e-12 * rng.normal(size=19)),                 # clustered
              (np.abs(rng.normal(size=25)) * 1e150, rng.normal(size=24) * 1e150),
              (rng.normal(size=25) * 1e-150, rng.normal(size=24) * 1e-150),
              (np.zeros(10), np.ones(9))]                                   # +-2 cos(j pi / 11)
    for a, b in cases:
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        ref = np.linalg.eigvalsh(T).max()
        got = orc.tridiag_max_eig(a, b)
        assert abs(got - ref) <= 1e-13 * max(np.abs(T).max(), 1e-300) * max(1, a.size), (a.size, got, ref)


def test_norm_estimate_rank_one(orc):
    # A = u v': the Krylov space is one-dimensional, so sigma = ||u|| ||v|| after one step (beta_1
    # is rounding-level, and the relative-change stop ends the process within two more steps)
    rng = np.random.default_rng(92)
    u, v = rng.normal(size=40), rng.normal(size=30)
    rp, ci, val = csr(np.outer(u, v))
    s, it = orc.norm_est(rp, ci, val, 30)
    assert it <= 3
    assert abs(s - np.linalg.norm(u) * np.linalg.norm(v)) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(v)
