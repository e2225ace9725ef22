"""Plain FP64 CPU reference of the learned warm start -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
use this module.  It shares no code with the CUDA library: features, the
3-layer network (features -> 512 -> 512 -> 1 per asset, ReLU), the per-instance
softmax, the mean-pooled dual head, the training loss and its gradient are
written out here from their definitions with numpy in FP64.

Pin: the analytic gradient is checked against central finite differences
(tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

HID = 512
FEAT = 16


def features(batch, rank):
    """Per-asset features of a portfolio batch (rows = assets of all instances)."""
    out = []
    for i in range(int(batch["batch_count"])):
        x0 = int(batch["x_off"][i])
        na = int(batch["n_assets"][i])
        k = int(rank[i])
        mu = -batch["c"][x0:x0 + na]
        d = batch["q_diag"][x0:x0 + na]
        F = batch["q_R"][:k, x0:x0 + na]
        f2 = (F * F).sum(axis=0)
        sig = batch["b"][int(batch["row_off"][i + 1]) - 1]
        f = np.zeros((na, FEAT))
        f[:, 0] = 20.0 * mu
        f[:, 1] = 20.0 * d
        f[:, 2] = 100.0 * f2
        f[:, 3] = 0.1 * mu / (d + f2)
        f[:, 4] = 50.0 * (mu - mu.mean())
        f[:, 5] = np.log(na) / 8.0
        f[:, 6] = k / 50.0
        f[:, 7] = 10.0 * sig
        rr = mu / (d + f2)
        f[:, 8] = (mu - mu.mean()) / (mu.std() + 1e-12)
        f[:, 9] = d / d.mean()
        f[:, 10] = f2 / f2.mean()
        f[:, 11] = rr / rr.max() if rr.max() > 0 else 0.0
        out.append(f)
    return np.concatenate(out, axis=0)


def forward(p, X, asset_off):
    """p: dict W1 (16x512), b1, W2 (512x512), b2, w3 (512), b3 (1), Wd (512x2), bd (2)."""
    Z1 = X @ p["W1"] + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"] + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    s = H2 @ p["w3"] + p["b3"][0]
    x0 = np.empty_like(s)
    count = len(asset_off) - 1
    pooled = np.zeros((count, HID))
    for i in range(count):
        a, e = int(asset_off[i]), int(asset_off[i + 1])
        z = np.exp(s[a:e] - s[a:e].max())
        x0[a:e] = z / z.sum()
        pooled[i] = H2[a:e].mean(axis=0)
    yd = pooled @ p["Wd"] + p["bd"]
    return dict(Z1=Z1, H1=H1, Z2=Z2, H2=H2, s=s, x0=x0, pooled=pooled, yd=yd)


def loss(f, xstar, ystar, asset_off, lam):
    L = 0.0
    for i in range(len(asset_off) - 1):
        a, e = int(asset_off[i]), int(asset_off[i + 1])
        L += (e - a) * np.sum((f["x0"][a:e] - xstar[a:e]) ** 2)
    return L + lam * np.sum((f["yd"] - ystar) ** 2)


def backward(p, X, f, xstar, ystar, asset_off, lam):
    """Gradient of `loss` with respect to every parameter (chain rule written out)."""
    count = len(asset_off) - 1
    ds = np.zeros_like(f["s"])
    dH2 = np.zeros_like(f["H2"])
    dyd = 2.0 * lam * (f["yd"] - ystar)
    g = {"Wd": f["pooled"].T @ dyd, "bd": dyd.sum(axis=0)}
    for i in range(count):
        a, e = int(asset_off[i]), int(asset_off[i + 1])
        n = e - a
        x = f["x0"][a:e]
        gx = 2.0 * n * (x - xstar[a:e])
        ds[a:e] = x * (gx - np.dot(x, gx))            # softmax Jacobian applied to gx
        dH2[a:e] += (p["Wd"] @ dyd[i]) / n             # mean pooling
    g["w3"] = f["H2"].T @ ds
    g["b3"] = np.array([ds.sum()])
    dH2 += np.outer(ds, p["w3"])
    dZ2 = dH2 * (f["Z2"] > 0)
    g["W2"] = f["H1"].T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"].T) * (f["Z1"] > 0)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return g
