"""Pins for the slice blocks of eq. fisher-conic and the market model built on them.

The paper stores each buyer's (z_i, 1, t_i) as a 3-D block whose middle entry is
held at one, with no affine row for it (Sec. 5.4, the coordinate and equation
counts after eq. fisher-conic).  The oracle's block types EXP1 / POW1 are those
slices, X_f = {(r, f, t): f e^{r/f} <= t} and {(x, f, z): x^a f^(1-a) >= |z|,
x >= 0}.  Their projections, support terms and whole solves are checked against
facts fixed without the oracle's slice code:

* the already-pinned metric projection onto the full cone with a huge weight on
  the middle coordinate converges to the slice projection as the weight grows;
* the normal-cone condition of the 2-D projection, and the variational
  inequality against dense samples of the slice (brute force);
* homogeneity X_f = f X_1;
* the support term in the KKT report against a dense scan of inf_{x in X} c'x;
* single-buyer markets, solved in closed form;
* the same market with explicit rows s_i = 1 over full cones (the other reading
  of the model) has the same optimum, and its optimal point makes the slice
  model's KKT report vanish.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import instances as I

EXP, POW, EXP1, POW1 = 4, 5, 7, 8


def _points(rng, k=40):
    out = []
    for _ in range(k):
        out.append(rng.normal(size=3) * rng.choice([0.1, 1.0, 4.0]))
    return out


def _metric(rng):
    return np.exp(rng.uniform(-1.5, 1.5, size=3))


def _in_exp_slice(u, f, tol):
    return abs(u[1] - f) <= tol and f * math.exp(u[0] / f) <= u[2] + tol * max(1.0, abs(u[2]))


def _in_pow_slice(u, f, a, tol):
    return abs(u[1] - f) <= tol and u[0] >= -tol and u[0] ** a * f ** (1 - a) + tol * max(1.0, abs(u[2])) >= abs(u[2]) \
        if u[0] >= 0 else False


# --------------------------------------------------------------------------- projections

@pytest.mark.parametrize("f", [1.0, 0.3, 2.5])
def test_inside_points_unchanged(orc, rng, f):
    for _ in range(30):
        r = rng.normal()
        t = f * math.exp(r / f) + abs(rng.normal())
        u = orc.proj_slice(EXP1, [r, 7.0, t], f=f, m=_metric(rng))
        assert u == pytest.approx([r, f, t], rel=1e-15, abs=1e-15)
        a = rng.uniform(0.2, 0.8)
        x = abs(rng.normal()) + 0.1
        z = (2 * rng.uniform() - 1) * x ** a * f ** (1 - a)
        u = orc.proj_slice(POW1, [x, -3.0, z], alpha=a, f=f, m=_metric(rng))
        assert u == pytest.approx([x, f, z], rel=1e-15, abs=1e-15)


@pytest.mark.parametrize("kind", [EXP1, POW1])
def test_limit_of_metric_cone_projection(orc, rng, kind):
    """Pi^{(m0, L, m2)}_K((r0, f, t0)) -> Pi^{(m0, m2)}_{X_f}(r0, t0) as L -> infinity (K the full cone)."""
    for r in _points(rng, 25):
        a = rng.uniform(0.25, 0.75)
        m = _metric(rng)
        f = float(rng.choice([1.0, 0.5, 2.0]))
        exact = orc.proj_slice(kind, r, alpha=a, f=f, m=m)
        errs = []
        for L in (1e4, 1e6, 1e8):
            mm = np.array([m[0], L, m[2]])
            u = orc.proj_block(EXP if kind == EXP1 else POW, [r[0], f, r[2]], alpha=a, m=mm)
            errs.append(np.max(np.abs(u - exact)) / max(1.0, np.max(np.abs(exact))))
        # the error of the penalised problem is O(1/L)
        assert errs[-1] <= 1e-6, (r, f, errs)
        assert errs[-1] <= errs[0] + 1e-12


def test_exp_slice_normal_cone(orc, rng):
    """Outside X_1: u = (a, 1, e^a) and M(r - u) = lam (e^a, 0, -1) with lam >= 0 (first two dims)."""
    n_out = 0
    for r in _points(rng, 60):
        m = _metric(rng)
        u = orc.proj_slice(EXP1, r, m=m)
        assert u[1] == 1.0
        if math.exp(r[0]) <= r[2]:
            continue
        n_out += 1
        assert u[2] == pytest.approx(math.exp(u[0]), rel=1e-14)
        g0, g2 = m[0] * (r[0] - u[0]), m[2] * (r[2] - u[2])
        lam = -g2
        assert lam >= -1e-12
        assert g0 == pytest.approx(lam * math.exp(u[0]), rel=1e-9, abs=1e-12)
    assert n_out > 10


def test_pow_slice_normal_cone(orc, rng):
    """Outside X_1 with z0 != 0: u = (x, 1, sign(z0) x^a), M(r - u) = lam (-a x^{a-1}, 0, sign z0), lam >= 0."""
    n_out = 0
    for r in _points(rng, 60):
        a = rng.uniform(0.2, 0.8)
        m = _metric(rng)
        u = orc.proj_slice(POW1, r, alpha=a, m=m)
        inside = r[0] >= 0 and r[0] ** a >= abs(r[2])
        if inside:
            continue
        n_out += 1
        x = u[0]
        assert x > 0
        assert abs(u[2]) == pytest.approx(x ** a, rel=1e-13)
        sg = math.copysign(1.0, r[2])
        lam = sg * m[2] * (r[2] - u[2])
        assert lam >= -1e-12
        assert m[0] * (r[0] - x) == pytest.approx(-lam * a * x ** (a - 1), rel=1e-8, abs=1e-12)
    assert n_out > 10


def _slice_samples(rng, kind, a, f, k=4000):
    """Dense samples of X_f: its boundary over a wide parameter range plus interior points."""
    if kind == EXP1:
        s = np.concatenate([np.linspace(-12, 6, k), rng.uniform(-12, 6, k)])
        t = f * np.exp(s) + np.concatenate([np.zeros(k), np.abs(rng.normal(size=k))])
        return np.stack([f * s, np.full_like(s, f), t], axis=1)
    x = np.concatenate([np.linspace(0, 30, k) ** 2 / 30, rng.uniform(0, 30, k)])
    bound = x ** a * f ** (1 - a)
    z = np.concatenate([np.ones(k), rng.uniform(-1, 1, k)]) * bound * np.where(rng.uniform(size=2 * k) < 0.5, 1, -1)
    return np.stack([x, np.full_like(x, f), z], axis=1)


@pytest.mark.parametrize("kind", [EXP1, POW1])
def test_variational_inequality_brute_force(orc, rng, kind):
    """<M(r - u), v - u> <= 0 for every sampled v in X_f, and u is at least as close as every sample."""
    for r in _points(rng, 20):
        a = rng.uniform(0.2, 0.8)
        f = float(rng.choice([1.0, 0.4, 3.0]))
        m = _metric(rng)
        u = orc.proj_slice(kind, r, alpha=a, f=f, m=m)
        V = _slice_samples(rng, kind, a, f)
        g = m * (np.asarray(r) - u)
        g[1] = 0.0   # the middle coordinate is fixed: no constraint on its multiplier
        vi = (V - u) @ g
        scale = np.linalg.norm(g) * (1.0 + np.linalg.norm(V - u, axis=1))
        assert np.all(vi <= 1e-9 * scale)
        du = np.sum(m[[0, 2]] * (u[[0, 2]] - np.asarray(r)[[0, 2]]) ** 2)
        dv = np.sum(m[[0, 2]] * (V[:, [0, 2]] - np.asarray(r)[[0, 2]]) ** 2, axis=1)
        assert du <= dv.min() * (1 + 1e-12) + 1e-14


@pytest.mark.parametrize("kind", [EXP1, POW1])
def test_homogeneity(orc, rng, kind):
    for r in _points(rng, 20):
        a = rng.uniform(0.2, 0.8)
        f = float(rng.uniform(0.1, 5.0))
        m = _metric(rng)
        u = orc.proj_slice(kind, r, alpha=a, f=f, m=m)
        u1 = orc.proj_slice(kind, np.asarray(r) / f, alpha=a, f=1.0, m=m)
        assert u == pytest.approx(f * u1, rel=1e-11, abs=1e-13)


def test_bad_arguments(orc):
    with pytest.raises(ValueError):
        orc.proj_slice(EXP1, [0.0, 1.0, 0.0], f=0.0)
    with pytest.raises(ValueError):
        orc.proj_slice(POW1, [0.0, 1.0, 0.0], alpha=1.0)
    with pytest.raises(ValueError):
        orc.proj_slice(EXP, [0.0, 1.0, 0.0])


# --------------------------------------------------------------------------- support term in the KKT report

def _one_block(kind, c, a=0.5, f=None):
    """n = 3 (one slice block), one empty row: the dual slack is c, so dobj = inf_{x in X} c'x."""
    inst = I.make_instance("slice", 1, 3, np.array([0, 0]), np.zeros(0, np.int64), np.zeros(0), np.asarray(c, float),
                           np.zeros(1), [kind], [0], [3], [a])
    if f is not None:
        inst["blk_fix"] = np.array([f])
    return inst


def _scan_inf(kind, c, a, f):
    if kind == EXP1:
        # inf over r of f (c0 r / f... ) on the boundary t = f e^{r/f}; interior points only add c2 * slack >= 0
        fun = lambda s: c[0] * f * s + c[2] * f * math.exp(s) + c[1] * f
        res = minimize_scalar(fun, bounds=(-60, 40), method="bounded", options={"xatol": 1e-12})
        grid = np.linspace(-60, 40, 200001)
        return min(res.fun, np.min(c[0] * f * grid + c[2] * f * np.exp(grid) + c[1] * f))
    fun = lambda x: c[0] * x - abs(c[2]) * x ** a * f ** (1 - a) + c[1] * f
    res = minimize_scalar(fun, bounds=(0, 1e6), method="bounded", options={"xatol": 1e-12})
    grid = np.linspace(0, 200, 400001)
    return min(res.fun, np.min(c[0] * grid - abs(c[2]) * grid ** a * f ** (1 - a) + c[1] * f))


@pytest.mark.parametrize("kind", [EXP1, POW1])
def test_support_term_against_scan(orc, rng, kind):
    for _ in range(12):
        a = rng.uniform(0.25, 0.75)
        f = float(rng.choice([1.0, 0.5, 2.0]))
        if kind == EXP1:
            c = np.array([-abs(rng.normal()) - 0.05, rng.normal(), abs(rng.normal()) + 0.05])
        else:
            c = np.array([abs(rng.normal()) + 0.2, rng.normal(), rng.normal()])
        rep = orc.kkt(_one_block(kind, c, a, f), np.array([0.0, f, 1.0]) if kind == EXP1 else np.array([1.0, f, 0.0]),
                      np.zeros(1))
        ref = _scan_inf(kind, c, a, f)
        assert rep["dobj"] == pytest.approx(ref, rel=1e-7, abs=1e-9)
        assert rep["norm_res_d"] == 0.0


def test_support_term_outside_domain(orc):
    # exp: c_r > 0 -> inf = -infinity along r -> -inf; the excess counts as dual residual
    rep = orc.kkt(_one_block(EXP1, [0.3, 0.0, 1.0]), np.array([0.0, 1.0, 1.0]), np.zeros(1))
    assert rep["norm_res_d"] == pytest.approx(0.3)
    rep = orc.kkt(_one_block(EXP1, [-0.5, 0.0, -0.25]), np.array([0.0, 1.0, 1.0]), np.zeros(1))
    assert rep["norm_res_d"] == pytest.approx(0.25)
    assert rep["dobj"] == -math.inf and rep["eps_g"] == 1.0
    # pow: c_x < 0 -> residual |c_x|; c_x = 0 with c_z != 0 -> -inf
    rep = orc.kkt(_one_block(POW1, [-0.4, 0.0, 0.0]), np.array([1.0, 1.0, 0.0]), np.zeros(1))
    assert rep["norm_res_d"] == pytest.approx(0.4)
    rep = orc.kkt(_one_block(POW1, [0.0, 0.0, 0.7]), np.array([1.0, 1.0, 0.0]), np.zeros(1))
    assert rep["dobj"] == -math.inf and rep["eps_g"] == 1.0


# --------------------------------------------------------------------------- whole solves

def _single_buyer_optimum(inst):
    """One buyer, one good of supply 1: x = 1, t = max(u, t_free), delta = t - u, objective delta - w z(t)
    with t_free = w (exp: z = log t, d/dt (t - w log t) = 0) or (w a)^{1/(1-a)} (pow: z = t^a)."""
    F = inst["fisher"]
    u, w = float(F["u"][0]), float(F["w"][0])
    if F["is_pow"][0]:
        a = float(F["alpha"][0])
        t = max(u, (w * a) ** (1.0 / (1.0 - a)))
        return (t - u) - w * t ** a
    t = max(u, w)
    return (t - u) - w * math.log(t)


@pytest.mark.parametrize("seed", [11, 12, 13, 14, 15, 16])
def test_single_buyer_closed_form(orc, seed):
    inst = I.fisher_market(n_buyers=1, n_goods=1, density=1.0, seed=seed)
    assert inst["m"] == 2 and inst["n"] == 5
    x, y, info = orc.solve(inst, tol=1e-10, max_iter=200000)
    assert info["status"] == 0
    ref = _single_buyer_optimum(inst)
    assert info["kkt"]["pobj"] == pytest.approx(ref, rel=1e-8, abs=1e-9)
    assert x[3] == pytest.approx(1.0, abs=1e-15)          # the fixed middle coordinate


@pytest.mark.parametrize("pow_fraction", [0.0, 0.5, 1.0])
def test_slice_model_matches_row_model(orc, pow_fraction):
    """Same market with explicit rows s_i = 1 over full cones: same optimum, and that optimum
    (restricted to the shared rows) makes the slice model's KKT report vanish."""
    kw = dict(n_buyers=40, n_goods=8, density=0.3, seed=2103, pow_fraction=pow_fraction)
    sl = I.fisher_market(fixed_middle=True, **kw)
    rw = I.fisher_market(fixed_middle=False, **kw)
    assert rw["m"] == sl["m"] + 40 and rw["n"] == sl["n"]
    xs, ys, infs = orc.solve(sl, tol=1e-9, max_iter=400000)
    xr, yr, infr = orc.solve(rw, tol=1e-9, max_iter=400000)
    assert infs["status"] == 0 and infr["status"] == 0
    assert infs["kkt"]["pobj"] == pytest.approx(infr["kkt"]["pobj"], rel=1e-7)
    rep = orc.kkt(sl, xr, yr[:sl["m"]])
    assert rep["rel_kkt"] <= 1e-7
    # a perturbed point is not optimal
    bad = orc.kkt(sl, xr, yr[:sl["m"]] * 1.01)
    assert bad["rel_kkt"] > 1e-5


def test_rescaled_cone_mode_with_slices(orc):
    inst = I.fisher_market(n_buyers=30, n_goods=6, density=0.4, seed=2104)
    _, _, a = orc.solve(inst, tol=1e-9, max_iter=400000)
    _, _, b = orc.solve(inst, tol=1e-9, max_iter=400000, rescaled_cones=1)
    assert a["status"] == 0 and b["status"] == 0
    assert a["kkt"]["pobj"] == pytest.approx(b["kkt"]["pobj"], rel=1e-7)


def test_nonpositive_fix_rejected(orc):
    inst = I.fisher_market(n_buyers=3, n_goods=2, density=1.0, seed=5)
    inst["blk_fix"] = np.array([1.0, 1.0, -1.0, 1.0])
    import ctypes
    P = orc._Prob(inst)
    o = orc.default_options()
    rc = orc.lib().orc_solve(P.ptr, ctypes.byref(o), None, None, None, None, None)
    assert rc == -1
