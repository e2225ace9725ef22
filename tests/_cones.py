"""Test-side cone geometry written independently of the oracle (numpy/scipy only).

Membership tests for each cone and its dual, and brute-force projections that
search the cone directly (constrained minimisation or a dense scan of the
boundary parameterisation) instead of solving the oracle's scalar equations.
"""
import math

import numpy as np
from scipy.optimize import minimize, minimize_scalar

FREE, NONNEG, SOC, RSOC, EXP, POW = 0, 1, 2, 3, 4, 5
EXP1, POW1 = 7, 8   # slices with the middle coordinate fixed at 1 (membership only)
E = math.e


_INTERIOR = {
    # a direction pointing into the interior of each cone (resp. its dual); membership with
    # tolerance tol is tested exactly at u + tol * scale * direction
    SOC: lambda d: np.r_[np.zeros(d - 1), 1.0],
    RSOC: lambda d: np.r_[np.zeros(d - 2), 1.0, 1.0],
    EXP: lambda d: np.array([-1.0, 1.0, 1.0]),
    POW: lambda d: np.array([1.0, 1.0, 0.0]),
    NONNEG: lambda d: np.ones(d),
    EXP1: lambda d: np.array([-1.0, 0.0, 1.0]),
    POW1: lambda d: np.array([1.0, 0.0, 0.0]),
}


def _in_cone_exact(t, u, alpha):
    if t == FREE:
        return True
    if t == NONNEG:
        return bool(np.all(u >= 0))
    if t == SOC:
        return bool(np.linalg.norm(u[:-1]) <= u[-1])
    if t == RSOC:
        v, s, w = u[:-2], u[-2], u[-1]
        return bool(s >= 0 and w >= 0 and v @ v <= 2 * s * w)
    if t == EXP:
        r, s, w = u
        if s > 0:
            return bool(w > 0 and r <= s * math.log(w / s))   # s exp(r/s) <= w without overflow
        return bool(r <= 0 and s == 0 and w >= 0)
    if t == POW:
        x, y, z = u
        if x < 0 or y < 0:
            return False
        return bool(x ** alpha * y ** (1 - alpha) >= abs(z))
    # the fixed coordinate comes back from the scaled variables as beta_b (col / beta_b) / col,
    # a few roundings from 1
    if t == EXP1:
        return bool(abs(u[1] - 1.0) <= 1e-14 and u[2] > 0 and u[0] <= math.log(u[2]))
    if t == POW1:
        return bool(abs(u[1] - 1.0) <= 1e-14 and u[0] >= 0 and u[0] ** alpha >= abs(u[2]))
    raise ValueError(t)


def _in_dual_exact(t, u, alpha):
    if t in (NONNEG, SOC, RSOC):
        return _in_cone_exact(t, u, alpha)
    if t == EXP:
        # K_exp* = cl{(a,b,c): a < 0, -a exp(b/a) <= e c}
        a, b, c = u
        if a < 0:
            return bool(c > 0 and math.log(-a) + b / a <= 1.0 + math.log(c))
        return bool(a == 0 and b >= 0 and c >= 0)
    if t == POW:
        p, q, w = u
        if p < 0 or q < 0:
            return False
        return bool((p / alpha) ** alpha * (q / (1 - alpha)) ** (1 - alpha) >= abs(w))
    raise ValueError(t)


def in_cone(t, u, alpha=0.0, tol=1e-9):
    u = np.asarray(u, float)
    if t == FREE:
        return True
    sc = tol * (1.0 + np.abs(u).max())
    return _in_cone_exact(t, u + sc * _INTERIOR[t](u.size), alpha)


def in_dual_cone(t, u, alpha=0.0, tol=1e-9):
    u = np.asarray(u, float)
    sc = tol * (1.0 + np.abs(u).max())
    if t == FREE:
        return bool(np.all(np.abs(u) <= sc))
    return _in_dual_exact(t, u + sc * _INTERIOR[t](u.size), alpha)


def certificate(t, r, u, m=None, alpha=0.0):
    """Residuals of the projection optimality conditions u in K, M(u - r) in K*, <u, M(u - r)> = 0."""
    r, u = np.asarray(r, float), np.asarray(u, float)
    m = np.ones_like(r) if m is None else np.asarray(m, float)
    g = m * (u - r)
    return in_cone(t, u, alpha, 1e-8), in_dual_cone(t, g, alpha, 1e-8), float(u @ g)


def _dist(u, r, m):
    d = u - r
    return float(np.sum(m * d * d))


def brute_exp(r, m):
    """Scan the smooth boundary eta (rho, 1, e^rho) with the optimal eta >= 0 for each rho,
    plus the face {s = 0, r <= 0, t >= 0} and the origin."""
    r = np.asarray(r, float)
    mr, ms, mt = m
    cands = [np.zeros(3), np.array([min(r[0], 0.0), 0.0, max(r[2], 0.0)])]
    if _in_cone_exact(EXP, r, 0.0):
        cands.append(r.copy())

    def best_on_ray(rho):
        a = np.array([rho, 1.0, math.exp(rho)])
        eta = max(0.0, float(np.sum(m * r * a)) / float(np.sum(m * a * a)))
        return eta * a

    def f(rho):
        return _dist(best_on_ray(rho), r, m)

    grid = np.concatenate([np.linspace(-40, 20, 60001), -np.logspace(1.7, 3, 200)])
    vals = np.array([f(x) for x in grid])
    i = int(np.argmin(vals))
    lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, grid.size - 1)]
    if lo > hi:
        lo, hi = hi, lo
    res = minimize_scalar(f, bounds=(lo, hi), method="bounded", options={"xatol": 1e-13})
    cands.append(best_on_ray(res.x))
    return min(cands, key=lambda u: _dist(u, r, m))


def brute_pow(r, m, alpha):
    """Minimise over the boundary (x, y, s x^a y^(1-a)), s = sign(r_z), from a grid of starts in
    log coordinates, plus the face z = 0 and the origin."""
    r = np.asarray(r, float)
    sgn = 1.0 if r[2] >= 0 else -1.0
    cands = [np.zeros(3), np.array([max(r[0], 0.0), max(r[1], 0.0), 0.0])]
    if _in_cone_exact(POW, r, alpha):
        cands.append(r.copy())

    def pt(p):
        x, y = math.exp(p[0]), math.exp(p[1])
        return np.array([x, y, sgn * x ** alpha * y ** (1 - alpha)])

    def f(p):
        return _dist(pt(p), r, m)

    scale = max(1.0, np.abs(r).max())
    best = None
    for lx in np.linspace(-12, math.log(4 * scale), 15):
        for ly in np.linspace(-12, math.log(4 * scale), 15):
            v = f((lx, ly))
            if best is None or v < best[0]:
                best = (v, (lx, ly))
    res = minimize(f, best[1], method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-16, "maxiter": 20000})
    cands.append(pt(res.x))
    return min(cands, key=lambda u: _dist(u, r, m))


def brute_soc_like(t, r, m):
    """SLSQP on the smooth description of SOC / RSOC from several starts."""
    r = np.asarray(r, float)
    d = r.size
    if t == SOC:
        cons = [{"type": "ineq", "fun": lambda u: u[-1]},
                {"type": "ineq", "fun": lambda u: u[-1] ** 2 - u[:-1] @ u[:-1]}]
    else:
        cons = [{"type": "ineq", "fun": lambda u: u[-2]}, {"type": "ineq", "fun": lambda u: u[-1]},
                {"type": "ineq", "fun": lambda u: 2 * u[-2] * u[-1] - u[:-2] @ u[:-2]}]
    starts = [np.abs(r) + 1.0, np.ones(d), r.copy()]
    best = np.zeros(d)
    for s0 in starts:
        res = minimize(lambda u: _dist(u, r, m), s0, jac=lambda u: 2 * m * (u - r), constraints=cons,
                       method="SLSQP", options={"ftol": 1e-15, "maxiter": 2000})
        u = res.x
        if in_cone(t, u, tol=1e-7) and _dist(u, r, m) < _dist(best, r, m):
            best = u
    return best


def soc_closed(r):
    """Euclidean SOC projection, closed form (App. A.2)."""
    r = np.asarray(r, float)
    v, t = r[:-1], r[-1]
    a = np.linalg.norm(v)
    if a <= t:
        return r.copy()
    if a <= -t:
        return np.zeros_like(r)
    return np.r_[(a + t) / (2 * a) * v, (a + t) / 2]


def rsoc_closed(r):
    """Euclidean RSOC projection through the orthogonal map U (App. A.3)."""
    r = np.asarray(r, float)
    h = 1 / math.sqrt(2)
    w = np.r_[r[:-2], (r[-2] - r[-1]) * h, (r[-2] + r[-1]) * h]
    p = soc_closed(w)
    return np.r_[p[:-2], (p[-2] + p[-1]) * h, (p[-1] - p[-2]) * h]
