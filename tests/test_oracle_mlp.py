"""Pins of the FP64 warm-start reference: analytic gradients against central finite
differences, the softmax start is feasible, and the features follow their definition."""
import numpy as np

import instances as I
from oracle import mlp as M


def _small_params(rng, hid=M.HID):
    return {"W1": rng.normal(size=(M.FEAT, hid)) * 0.3, "b1": rng.normal(size=hid) * 0.1,
            "W2": rng.normal(size=(hid, hid)) * 0.05, "b2": rng.normal(size=hid) * 0.1,
            "w3": rng.normal(size=hid) * 0.1, "b3": np.array([0.05]),
            "Wd": rng.normal(size=(hid, 2)) * 0.1, "bd": np.array([0.01, -0.02])}


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    b = I.portfolio_batch(count=3, n_range=(4, 7), k_range=(2, 3), seed=91)
    rank = b["n_factors"]
    X = M.features(b, rank)
    off = np.concatenate([[0], np.cumsum(b["n_assets"])])
    p = _small_params(rng)
    xs = np.concatenate([rng.dirichlet(np.ones(int(n))) for n in b["n_assets"]])
    ys = rng.normal(size=(3, 2))
    lam = 0.7
    f = M.forward(p, X, off)
    g = M.backward(p, X, f, xs, ys, off, lam)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3", "b3", "Wd", "bd"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(M.forward(p, X, off), xs, ys, off, lam)
            flat[idx] = old - h
            lm = M.loss(M.forward(p, X, off), xs, ys, off, lam)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * (1 + abs(fd)), (name, idx, fd, an)


def test_softmax_start_is_feasible_and_features_by_definition():
    rng = np.random.default_rng(4)
    b = I.portfolio_batch(count=4, n_range=(5, 9), k_range=(2, 4), seed=92)
    X = M.features(b, b["n_factors"])
    off = np.concatenate([[0], np.cumsum(b["n_assets"])])
    f = M.forward(_small_params(rng), X, off)
    for i in range(4):
        x = f["x0"][off[i]:off[i + 1]]
        assert np.all(x > 0) and abs(x.sum() - 1) <= 1e-12
    # feature 0 is 20 mu, feature 2 is 100 |F_j|^2 for the first asset of instance 0
    mu0 = -b["c"][0]
    F0 = b["q_R"][:int(b["n_factors"][0]), 0]
    assert abs(X[0, 0] - 20 * mu0) <= 1e-12 and abs(X[0, 2] - 100 * F0 @ F0) <= 1e-12
