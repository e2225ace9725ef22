"""Pins for the oracle's cone projections (App. A of the paper).

Each projection is checked against facts that do not depend on the oracle's
own root-finding:
  * the optimality certificate u in K, M(u - r) in K*, <u, M(u - r)> = 0,
    which characterises Pi^M_K(r) uniquely (App. A, opening paragraph);
  * brute-force search of the cone (constrained minimisation or a dense scan of
    the boundary parameterisation) on small inputs;
  * closed forms (box / nonnegative, SOC, RSOC through the orthogonal map U);
  * agreement of independent code paths (M-norm routines at M = I against the
    Euclidean ones);
  * the Moreau decomposition r = Pi_K(r) - Pi_K*(-r) for the self-dual cones;
  * the special cases printed in App. A (exp face, power r_z = 0, RSOC singular).
"""
import math

import numpy as np
import pytest

import _cones as G

TYPES = [(G.SOC, 5), (G.RSOC, 6), (G.EXP, 3), (G.POW, 3)]


def _samples(rng, t, d, k):
    out = []
    for i in range(k):
        scale = 10.0 ** rng.uniform(-2, 2)
        r = rng.normal(size=d) * scale
        if i % 7 == 0:
            r[-1] = abs(r[-1])
        if t == G.EXP and i % 5 == 1:
            r[0], r[1] = abs(r[0]), abs(r[1])          # forces the root-finding branch
        if t == G.EXP and i % 5 == 2:
            r[1] = abs(r[1])
        out.append(r)
    return out


def _metric(rng, d, wide=False):
    return np.exp(rng.normal(size=d) * (2.0 if wide else 0.7))


def _pythagoras(u, ub, r, m, tol):
    """For the projection u of r onto a closed convex set and any feasible point ub:
    ||ub - r||_M^2 >= ||u - r||_M^2 + ||ub - u||_M^2.  Holds whether or not the brute-force
    search converged; if it did, it forces ub close to u."""
    du = float(np.sum(m * (u - r) ** 2))
    db = float(np.sum(m * (ub - r) ** 2))
    gap = float(np.sum(m * (ub - u) ** 2))
    scale = 1.0 + float(np.sum(m * r * r))
    assert du <= db + tol * scale, (du, db)
    assert gap <= max(db - du, 0.0) + tol * scale, (gap, db - du)


@pytest.mark.parametrize("t,d", TYPES)
@pytest.mark.parametrize("metric", ["euclid", "mnorm", "mnorm_wide"])
def test_certificate(orc, rng, t, d, metric):
    for r in _samples(rng, t, d, 300):
        alpha = rng.uniform(0.15, 0.85)
        m = None if metric == "euclid" else _metric(rng, d, metric == "mnorm_wide")
        u = orc.proj_block(t, r, alpha=alpha, m=m)
        ink, indual, comp = G.certificate(t, r, u, m, alpha)
        mm = np.ones(d) if m is None else m
        scale = 1.0 + float(np.abs(mm * r).max()) * (1.0 + float(np.abs(r).max()))
        assert ink, (t, r, m, u)
        assert indual, (t, r, m, u)
        assert abs(comp) <= 1e-9 * scale, (t, r, m, u, comp)


@pytest.mark.parametrize("metric", ["euclid", "mnorm", "mnorm_wide"])
def test_exp_brute_force(orc, rng, metric):
    for _ in range(25):
        r = rng.normal(size=3) * 10.0 ** rng.uniform(-1, 1)
        m = np.ones(3) if metric == "euclid" else _metric(rng, 3, metric == "mnorm_wide")
        u = orc.proj_block(G.EXP, r, m=None if metric == "euclid" else m)
        ub = G.brute_exp(r, m)
        _pythagoras(u, ub, r, m, 1e-10)


@pytest.mark.parametrize("metric", ["euclid", "mnorm"])
def test_pow_brute_force(orc, rng, metric):
    for _ in range(20):
        r = rng.normal(size=3) * 10.0 ** rng.uniform(-1, 1)
        alpha = rng.uniform(0.2, 0.8)
        m = np.ones(3) if metric == "euclid" else _metric(rng, 3)
        u = orc.proj_block(G.POW, r, alpha=alpha, m=None if metric == "euclid" else m)
        ub = G.brute_pow(r, m, alpha)
        _pythagoras(u, ub, r, m, 1e-9)


@pytest.mark.parametrize("t,d", [(G.SOC, 4), (G.RSOC, 5)])
def test_soc_rsoc_brute_force(orc, rng, t, d):
    for _ in range(25):
        r = rng.normal(size=d) * 3
        m = _metric(rng, d)
        u = orc.proj_block(t, r, m=m)
        ub = G.brute_soc_like(t, r, m)
        _pythagoras(u, ub, r, m, 1e-7)


def test_soc_closed_form_and_moreau(orc, rng):
    for _ in range(200):
        d = int(rng.integers(2, 12))
        r = rng.normal(size=d) * 3
        u = orc.proj_block(G.SOC, r)
        v, t = r[:-1], r[-1]
        a = np.linalg.norm(v)
        if a <= t:
            ref = r
        elif a <= -t:
            ref = np.zeros(d)
        else:
            ref = np.concatenate([(a + t) / (2 * a) * v, [(a + t) / 2]])
        assert np.allclose(u, ref, rtol=1e-14, atol=1e-14)
        # SOC is self-dual: r = Pi_K(r) - Pi_K(-r)
        assert np.allclose(r, u - orc.proj_block(G.SOC, -r), atol=1e-13)
        # M-norm routine at M = I (bisection path) agrees with the closed form
        assert np.allclose(orc.proj_block(G.SOC, r, m=np.ones(d)), ref, atol=1e-12 * (1 + np.abs(r).max()))


def test_rsoc_euclid_vs_mnorm_identity_and_moreau(orc, rng):
    for _ in range(200):
        d = int(rng.integers(3, 10))
        r = rng.normal(size=d) * 3
        u = orc.proj_block(G.RSOC, r)                  # through U and the SOC closed form
        u2 = orc.proj_block(G.RSOC, r, m=np.ones(d))   # through the xi root (independent path)
        assert np.allclose(u, u2, atol=1e-10 * (1 + np.abs(r).max()))
        assert np.allclose(r, u - orc.proj_block(G.RSOC, -r), atol=1e-12 * (1 + np.abs(r).max()))


def test_exp_euclid_vs_mnorm_identity(orc, rng):
    for _ in range(300):
        r = rng.normal(size=3) * 10.0 ** rng.uniform(-2, 2)
        u = orc.proj_block(G.EXP, r)
        u2 = orc.proj_block(G.EXP, r, m=np.ones(3))
        assert np.allclose(u, u2, atol=1e-10 * (1 + np.abs(r).max()))


def test_nonneg_box(orc, rng):
    r = rng.normal(size=50)
    m = _metric(rng, 50)
    assert np.array_equal(orc.proj_block(G.NONNEG, r), np.maximum(r, 0))
    assert np.array_equal(orc.proj_block(G.NONNEG, r, m=m), np.maximum(r, 0))   # metric independent (App. A.1)
    assert np.array_equal(orc.proj_block(G.FREE, r), r)


def test_trivial_cases(orc, rng):
    # in K -> itself; -M r in K* -> 0 (App. A opening paragraph)
    assert np.allclose(orc.proj_block(G.SOC, np.array([0.3, 0.4, 1.0])), [0.3, 0.4, 1.0])
    assert np.allclose(orc.proj_block(G.SOC, np.array([0.3, 0.4, -1.0])), 0)
    assert np.allclose(orc.proj_block(G.EXP, np.array([0.0, 1.0, 2.0])), [0.0, 1.0, 2.0])
    assert np.allclose(orc.proj_block(G.EXP, np.array([1.0, -1.0, -3.0])), 0)
    # exp face case r0 <= 0, s0 <= 0 -> (r0, 0, max(t0, 0)) in both metrics (App. A.4)
    for r in ([-1.0, -2.0, 3.0], [-1.0, -0.5, -3.0], [-0.2, -1e-3, 0.5]):
        r = np.array(r)
        ref = np.array([r[0], 0.0, max(r[2], 0.0)])
        if not G.in_dual_cone(G.EXP, -r):
            assert np.allclose(orc.proj_block(G.EXP, r), ref)
            assert np.allclose(orc.proj_block(G.EXP, r, m=np.array([2.0, 0.3, 5.0])), ref)
    # power cone r_z = 0 -> (max(rx,0), max(ry,0), 0) in both metrics (App. A.5)
    for rx, ry in [(-1.0, 2.0), (1.5, -0.5), (0.7, 0.9)]:
        r = np.array([rx, ry, 0.0])
        ref = np.array([max(rx, 0), max(ry, 0), 0.0])
        assert np.allclose(orc.proj_block(G.POW, r, alpha=0.3), ref)
        assert np.allclose(orc.proj_block(G.POW, r, alpha=0.3, m=np.array([2.0, 0.5, 3.0])), ref)


def test_rsoc_singular_case(orc, rng):
    # consistent right-hand side sqrt(ms) rs + sqrt(mt) rt = 0 (eq. rsoc-metric-singular-projection):
    # the closed form must satisfy the certificate and match the limit of nearby inputs
    for _ in range(50):
        d = 5
        m = _metric(rng, d)
        r = rng.normal(size=d)
        r[-1] = -math.sqrt(m[-2]) * r[-2] / math.sqrt(m[-1])
        u = orc.proj_block(G.RSOC, r, m=m)
        ink, indual, comp = G.certificate(G.RSOC, r, u, m)
        assert ink and indual and abs(comp) < 1e-9 * (1 + np.abs(r).max()) ** 2
        rp = r.copy()
        rp[-1] += 1e-7
        assert np.allclose(orc.proj_block(G.RSOC, rp, m=m), u, atol=1e-5)


def test_case_boundaries_continuity(orc):
    # at the case boundaries the branches agree (inputs +-1 ulp apart)
    for t, r in [(G.SOC, [3.0, 4.0, 5.0]), (G.SOC, [3.0, 4.0, -5.0]),
                 (G.EXP, [1.0, 1.0, math.e]), (G.POW, [1.0, 1.0, 1.0])]:
        r = np.array(r, float)
        lo = r.copy()
        lo[-1] = np.nextafter(lo[-1], -np.inf)
        hi = r.copy()
        hi[-1] = np.nextafter(hi[-1], np.inf)
        a = orc.proj_block(t, lo, alpha=0.5)
        b = orc.proj_block(t, hi, alpha=0.5)
        assert np.allclose(a, b, atol=1e-7), (t, a, b)


def test_power_bracket_limits(orc):
    # Prop. power-cone-bisection: the unique zero lies in (0, R); the projection's |u_z| < R
    rng = np.random.default_rng(3)
    for _ in range(200):
        r = rng.normal(size=3) * 2
        alpha = rng.uniform(0.1, 0.9)
        m = np.exp(rng.normal(size=3))
        u = orc.proj_block(G.POW, r, alpha=alpha, m=m)
        if np.abs(u).max() > 0 and not G.in_cone(G.POW, r, alpha):
            assert abs(u[2]) < abs(r[2]) + 1e-15
            assert np.sign(u[2]) == np.sign(r[2]) or u[2] == 0


def test_dual_cone_pairing(rng):
    # the (test-side) dual descriptions give <x, y> >= 0 on sampled pairs; the exponential
    # dual is not printed in the paper, so it is checked numerically here
    for t, d in [(G.EXP, 3), (G.POW, 3)]:
        xs, ys = [], []
        while len(xs) < 300 or len(ys) < 300:
            v = rng.normal(size=d) * 3
            a = rng.uniform(0.2, 0.8)
            if G.in_cone(t, v, 0.4, 0):
                xs.append(v)
            if G.in_dual_cone(t, v, 0.4, 0):
                ys.append(v)
        X, Y = np.array(xs[:300]), np.array(ys[:300])
        assert (X @ Y.T).min() >= -1e-12


def _random_in_cone(rng, t, d, alpha):
    """Random points of K: interior points and points on its boundary."""
    if t == G.SOC:
        v = rng.normal(size=d - 1) * 3
        return np.r_[v, np.linalg.norm(v) + abs(rng.normal()) * rng.integers(0, 2)]
    if t == G.RSOC:
        v = rng.normal(size=d - 2) * 3
        s_ = abs(rng.normal()) * 3 + 1e-3
        return np.r_[v, s_, v @ v / (2 * s_) + abs(rng.normal()) * rng.integers(0, 2)]
    if t == G.EXP:
        s_ = abs(rng.normal()) * 3 + 1e-3
        r_ = min(rng.normal() * 3, 30.0 * s_)
        return np.array([r_, s_, s_ * np.exp(r_ / s_) + abs(rng.normal()) * rng.integers(0, 2)])
    if t == G.POW:
        x, y = abs(rng.normal(size=2)) * 3
        g = x ** alpha * y ** (1 - alpha)
        return np.array([x, y, g * rng.uniform(-1, 1) ** rng.integers(0, 2)])


@pytest.mark.parametrize("t,d", TYPES)
def test_variational_inequality(orc, rng, t, d):
    """<M(r - u), z - u> <= 0 for every z in K characterises u = Pi^M_K(r) (u in K)."""
    for _ in range(60):
        r = rng.normal(size=d) * 10.0 ** rng.uniform(-1, 1)
        alpha = rng.uniform(0.2, 0.8)
        m = _metric(rng, d)
        u = orc.proj_block(t, r, alpha=alpha, m=m)
        Z = np.array([_random_in_cone(rng, t, d, alpha) for _ in range(200)])
        vi = (Z - u) @ (m * (r - u))
        scale = (1 + np.abs(r).max()) * (1 + np.abs(Z).max()) * (1 + m.max())
        assert vi.max() <= 1e-9 * scale, (t, r, m, u, vi.max())
