"""Pins of the oracle's rescaled-cone mode (Sec. 4.2.2, eq. scaling-induced-metric):
the Ruiz and Pock-Chambolle column factors stay coordinatewise on cone blocks. Each
block then becomes S_j K_j, and its projection is S Pi_K^{S m S}(S^-1 r).

* The scaled projection satisfies the Moreau certificate of the set S K in the metric m.
  That is u in S K, S M (u - r) in K*, and <M (u - r), u> = 0, with (S K)* = S^-1 K*.
  This is checked for every cone family, Euclidean and metric.
* The rescaled-cone mode really leaves factors coordinatewise inside cone blocks, and
  the cone-preserving mode makes them constant per block.
* Whole solves in the rescaled-cone mode meet the KKT conditions of the original
  problem:
  - min 1/2||x - p||^2 with a'x = beta over one cone equals Pi_K(p + lam a), where lam
    is the root of a'Pi_K(p + lam a) = beta, found by bisection;
  - the mixed SOC/RSOC QP gives the unique optimum of the cone-preserving mode;
  - the exp/pow market gives the same objective as the cone-preserving mode.
"""
import numpy as np
import pytest

import _cones as G
import instances as I

SOC, RSOC, EXP, POW = I.CONE_SOC, I.CONE_RSOC, I.CONE_EXP, I.CONE_POW


def _cases(rng):
    for t, d in ((SOC, 6), (RSOC, 6), (EXP, 3), (POW, 3)):
        for _ in range(25):
            yield t, d, (rng.uniform(0.2, 0.8) if t == POW else 0.0)


@pytest.mark.parametrize("metric", [False, True])
def test_scaled_projection_certificate(orc, metric):
    rng = np.random.default_rng(31 + metric)
    for t, d, al in _cases(rng):
        r = rng.normal(size=d) * rng.choice([0.1, 1.0, 10.0])
        sc = np.exp(rng.uniform(-1.5, 1.5, d))
        m = np.exp(rng.uniform(-1.0, 1.0, d)) if metric else None
        u = orc.proj_block_scaled(t, sc, r, alpha=al, m=m)
        M = np.ones(d) if m is None else m
        # u in S K, S M (u - r) in K*, <M (u - r), u> = 0: the certificate of w = u / sc as the
        # projection of r / sc onto K in the metric M sc^2, checked by the test-side cone tests
        ink, indual, comp = G.certificate(t, r / sc, u / sc, M * sc * sc, al)
        scale = 1.0 + np.abs(M * r).max() * (1.0 + np.abs(r).max())
        assert ink and indual, (t, r, sc, m, u)
        assert abs(comp) <= 1e-9 * scale, (t, comp)
        # optimality against feasible points of S K (samples of the cone, scaled)
        base = ((u - r) * M) @ (u - r)
        for _ in range(50):
            w = orc.proj_block(t, rng.normal(size=d) * scale, alpha=al)
            v = sc * w
            assert ((v - r) * M) @ (v - r) >= base - 1e-9 * scale * scale * M.max()


def _one_cone_row(t, d, al, rng):
    """min 1/2||x - p||^2 s.t. a'x = beta, x in K (one cone block); the entries of a spread
    over two decades so the column factors differ inside the block."""
    a = rng.choice([-1.0, 1.0], d) * 10.0 ** rng.uniform(-1.0, 1.0, d)
    x0 = I.interior_point(I.Stream(int(rng.integers(1 << 30))), np.array([t]), np.array([0]), np.array([d]),
                          np.array([al]), d)
    p = rng.normal(size=d)
    beta = float(a @ x0)
    rp, ci, v = I._coo_to_csr(1, d, np.zeros(d, np.int64), np.arange(d), a)
    bt, bs, bd, ba = I.blocks_from_list([(t, d, al)])
    inst = I.make_instance("one", 1, d, rp, ci, v, -p, np.array([beta]), bt, bs, bd, ba, q_diag=np.ones(d))
    return inst, a, p, beta


def _bisect_reference(orc, t, al, a, p, beta):
    f = lambda lam: a @ orc.proj_block(t, p + lam * a, alpha=al) - beta
    lo, hi = -1.0, 1.0
    while f(lo) > 0:
        lo *= 2
    while f(hi) < 0:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return orc.proj_block(t, p + 0.5 * (lo + hi) * a, alpha=al)


@pytest.mark.parametrize("t,d", [(SOC, 6), (RSOC, 6), (EXP, 3), (POW, 3)])
def test_one_row_over_one_cone(orc, t, d):
    rng = np.random.default_rng(40 + t)
    al = 0.35 if t == POW else 0.0
    inst, a, p, beta = _one_cone_row(t, d, al, rng)
    sc = orc.rescale(inst, rescaled_cones=1)["col"]
    assert sc.max() / sc.min() > 1.5      # the block's factors are not aggregated
    ref = _bisect_reference(orc, t, al, a, p, beta)
    x, y, info = orc.solve(inst, tol=1e-10, max_iter=20000, rescaled_cones=1)
    assert info["status"] == 0
    assert np.abs(x - ref).max() <= 1e-6 * (1 + np.abs(ref).max())


def test_modes_scale_as_specified(orc):
    inst = I.small_config(2)
    c0 = orc.rescale(inst)["col"]
    c1 = orc.rescale(inst, rescaled_cones=1)["col"]
    spread0, spread1 = [], []
    for t, s, d in zip(inst["blk_type"], inst["blk_start"], inst["blk_dim"]):
        if t in (SOC, RSOC):
            seg0, seg1 = c0[s:s + d], c1[s:s + d]
            spread0.append(seg0.max() / seg0.min())
            spread1.append(seg1.max() / seg1.min())
    assert max(spread0) == 1.0
    assert np.median(spread1) > 1.2


def test_mixed_cones_same_optimum(orc):
    inst = I.small_config(2)     # Q = diag + R'R positive definite: x* unique
    x0, y0, i0 = orc.solve(inst, tol=1e-8, max_iter=20000)
    x1, y1, i1 = orc.solve(inst, tol=1e-8, max_iter=20000, rescaled_cones=1)
    assert i0["status"] == 0 and i1["status"] == 0
    assert orc.kkt(inst, x1, y1)["rel_kkt"] <= 1e-8
    assert np.abs(x1 - x0).max() <= 1e-4 * (1 + np.abs(x0).max())


def test_market_same_objective(orc):
    inst = I.small_config(3)     # exp and pow blocks, diagonal-Q path
    _, _, i0 = orc.solve(inst, tol=1e-6, max_iter=20000)
    x1, y1, i1 = orc.solve(inst, tol=1e-6, max_iter=20000, rescaled_cones=1)
    assert i0["status"] == 0 and i1["status"] == 0
    rep = orc.kkt(inst, x1, y1)
    assert rep["rel_kkt"] <= 1e-6
    assert abs(rep["pobj"] - i0["kkt"]["pobj"]) <= 1e-5 * (1 + abs(i0["kkt"]["pobj"]))
