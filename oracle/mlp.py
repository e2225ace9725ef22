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


def layer(Hin, W, b):
    """One hidden layer: Z = Hin W + b, H = max(Z, 0)."""
    Z = Hin @ W + b
    return Z, np.maximum(Z, 0.0)


def head_forward(p, H2, asset_off):
    """Scores s = H2 w3 + b3, per-instance softmax x0, mean-pooled H2 and the dual head yd."""
    s = H2 @ p["w3"] + p["b3"][0]
    x0 = np.empty_like(s)
    count = len(asset_off) - 1
    pooled = np.zeros((count, H2.shape[1]))
    for i in range(count):
        a, e = int(asset_off[i]), int(asset_off[i + 1])
        z = np.exp(s[a:e] - s[a:e].max())
        x0[a:e] = z / z.sum()
        pooled[i] = H2[a:e].mean(axis=0)
    yd = pooled @ p["Wd"] + p["bd"]
    return dict(s=s, x0=x0, pooled=pooled, yd=yd)


def forward(p, X, asset_off):
    """p: dict W1 (16x512), b1, W2 (512x512), b2, w3 (512), b3 (1), Wd (512x2), bd (2)."""
    Z1, H1 = layer(X, p["W1"], p["b1"])
    Z2, H2 = layer(H1, p["W2"], p["b2"])
    f = dict(Z1=Z1, H1=H1, Z2=Z2, H2=H2)
    f.update(head_forward(p, H2, asset_off))
    return f


def loss(f, xstar, ystar, asset_off, lam):
    L = 0.0
    for i in range(len(asset_off) - 1):
        a, e = int(asset_off[i]), int(asset_off[i + 1])
        L += (e - a) * np.sum((f["x0"][a:e] - xstar[a:e]) ** 2)
    return L + lam * np.sum((f["yd"] - ystar) ** 2)


def head_input_grad(p, ds, dyd, asset_off):
    """Derivative of the loss with respect to the head's input H2 (before the ReLU mask of
    layer 2): ds w3' from the scores plus Wd dyd / n_i from the mean pooling of instance i."""
    dH2 = np.outer(ds, p["w3"])
    for i in range(len(asset_off) - 1):
        a, e = int(asset_off[i]), int(asset_off[i + 1])
        dH2[a:e] += (p["Wd"] @ dyd[i]) / (e - a)
    return dH2


def head_backward(p, f, xstar, ystar, asset_off, lam):
    """Derivatives of `loss` through the head: ds (scores), dyd (dual head), dH2 (the head's
    input, before the ReLU mask of layer 2) and the head's parameter gradients."""
    count = len(asset_off) - 1
    ds = np.zeros_like(f["s"])
    dyd = 2.0 * lam * (f["yd"] - ystar)
    g = {"Wd": f["pooled"].T @ dyd, "bd": dyd.sum(axis=0)}
    for i in range(count):
        a, e = int(asset_off[i]), int(asset_off[i + 1])
        n = e - a
        x = f["x0"][a:e]
        gx = 2.0 * n * (x - xstar[a:e])
        ds[a:e] = x * (gx - np.dot(x, gx))            # softmax Jacobian applied to gx
    g["w3"] = f["H2"].T @ ds
    g["b3"] = np.array([ds.sum()])
    return ds, dyd, head_input_grad(p, ds, dyd, asset_off), g


def layer_backward(Hin, dZ, W=None, mask_in=None):
    """Gradients of a layer Z = Hin W + b from dZ: dW = Hin' dZ, db = sum of dZ over rows, and
    (with W) the input's derivative dZ W' masked by the previous ReLU (mask_in: Z_in > 0)."""
    dW, db = Hin.T @ dZ, dZ.sum(axis=0)
    dHin = None
    if W is not None:
        dHin = dZ @ W.T
        if mask_in is not None:
            dHin = dHin * mask_in
    return dW, db, dHin


def backward(p, X, f, xstar, ystar, asset_off, lam):
    """Gradient of `loss` with respect to every parameter (chain rule written out)."""
    ds, dyd, dH2, g = head_backward(p, f, xstar, ystar, asset_off, lam)
    dZ2 = dH2 * (f["Z2"] > 0)
    g["W2"], g["b2"], dZ1 = layer_backward(f["H1"], dZ2, p["W2"], f["Z1"] > 0)
    g["W1"], g["b1"], _ = layer_backward(X, dZ1)
    return g
