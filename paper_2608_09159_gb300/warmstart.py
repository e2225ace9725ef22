"""Learned warm start for batches of portfolio QPs (entry points of include/cqp_mlp.h).

A 3-layer MLP (features -> 512 -> 512 -> 1 per asset, ReLU, BF16 weights and
activations, FP32 accumulation and master weights) proposes the start (x0, y0)
of cqp_solve_batch: x0 is the softmax of the asset scores within each instance
(so 1'x0 = 1, x0 >= 0) completed by w_F = F'x0, w_D = D^(1/2) x0, t = sigma_bar;
a dual head predicts the budget-row and risk-row duals, which seed those two rows
of y0 (the other duals start at zero, which measured best).  The
network is trained on solutions of the batched solver.  Device memory is held
in torch tensors; every computation is one of the library's kernels, called
through the C ABI.  The solver is unchanged and a cold start stays available.
"""
from __future__ import annotations

import math

import numpy as np

from . import (BatchSolver, cqp_adam_step, cqp_gemm_bf16, cqp_relu_backward_bf16, cqp_transpose_bf16, cqp_ws_features,
               cqp_ws_head_backward, cqp_ws_head_forward, cqp_ws_loss, cqp_ws_start)

HID = 512
FEAT = 16
YB_SCALE = 20.0          # the budget dual is predicted as YB_SCALE * y_budget
PARAMS = ("W1", "b1", "W2", "b2", "w3", "b3", "Wd", "bd")


def _p(t):
    return None if t is None else t.data_ptr()


_DEVICE_KEYS = {"a_rowptr": np.int64, "a_colind": np.int32, "a_val": np.float64, "c": np.float64, "b": np.float64,
                "q_diag": np.float64, "q_R": np.float64, "q_D": np.float64, "blk_type": np.int32,
                "blk_start": np.int64, "blk_dim": np.int64, "blk_alpha": np.float64}


def _cuda(a, dt):
    import torch
    if hasattr(a, "data_ptr"):
        return a
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def to_device(batch):
    """The batch with its problem arrays copied to the device once (shared by the solver
    and the warm start)."""
    out = dict(batch)
    for k, dt in _DEVICE_KEYS.items():
        if batch.get(k) is not None:
            out[k] = _cuda(batch[k], dt)
    return out


class BatchDevice:
    """Device copies of the arrays of a portfolio batch that the warm start reads
    (arrays that are already CUDA tensors are used in place)."""

    def __init__(self, batch):
        cuda = _cuda
        self.count = int(batch["batch_count"])
        self.n, self.m = int(batch["n"]), int(batch["m"])
        na = np.asarray(batch["n_assets"], dtype=np.int64)
        self.asset_off_h = np.concatenate([[0], np.cumsum(na)]).astype(np.int64)
        self.rows = int(self.asset_off_h[-1])
        self.x_off = cuda(batch["x_off"], np.int64)
        self.row_off = cuda(batch["row_off"], np.int64)
        self.n_assets = cuda(na, np.int64)
        self.asset_off = cuda(self.asset_off_h, np.int64)
        self.rank = cuda(batch["n_factors"], np.int32)
        self.c = cuda(batch["c"], np.float64)
        self.q = cuda(batch["q_diag"], np.float64)
        self.b = cuda(batch["b"], np.float64)
        self.R = cuda(batch["q_R"], np.float64)
        self.ldr = self.n

    def features(self):
        import torch
        X = torch.empty(self.rows, FEAT, dtype=torch.bfloat16, device="cuda")
        cqp_ws_features(self.count, _p(self.x_off), _p(self.n_assets), _p(self.asset_off), _p(self.row_off),
                        _p(self.rank), _p(self.c), _p(self.q), _p(self.R), self.ldr, _p(self.b), _p(X))
        return X


def targets(batch, x, y):
    """Training targets of a solved batch: the asset weights (FP32, rows) and the
    scaled budget and risk duals (count x 2)."""
    xo, ro, na = batch["x_off"], batch["row_off"], batch["n_assets"]
    xs = np.concatenate([x[int(xo[i]):int(xo[i]) + int(na[i])] for i in range(int(batch["batch_count"]))])
    ys = np.stack([YB_SCALE * y[ro[:-1]], y[ro[1:] - 1]], axis=1)
    return xs.astype(np.float32), ys.astype(np.float32)


class WarmStartNet:
    def __init__(self, seed: int = 0):
        import torch
        self.torch = torch
        g = torch.Generator().manual_seed(seed)
        rn = lambda shape, std: (torch.randn(*shape, generator=g, dtype=torch.float64) * std).float().cuda()
        z = lambda *shape: torch.zeros(*shape, dtype=torch.float32, device="cuda")
        self.p = {"W1": rn((FEAT, HID), math.sqrt(2.0 / 8)), "b1": z(HID),
                  "W2": rn((HID, HID), math.sqrt(2.0 / HID)), "b2": z(HID),
                  "w3": rn((HID,), 0.01), "b3": z(1), "Wd": z(HID, 2), "bd": z(2)}
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.bf = {k: torch.empty(self.p[k].shape, dtype=torch.bfloat16, device="cuda") for k in ("W1", "W2")}
        # W2' in BF16: layer 2's forward product H1 W2 = H1 (W2')' takes the tensor-memory GEMM
        # (A times the transpose of a K-contiguous B)
        self.w2t = torch.empty(HID, HID, dtype=torch.bfloat16, device="cuda")
        self.step = 0
        # BF16 copies of the initial weights through the Adam kernel with a zero step
        for k in ("W1", "W2"):
            cqp_adam_step(self.p[k].numel(), _p(self.p[k]), _p(self.g[k]), _p(self.m[k]), _p(self.v[k]), 0.0, 0.9,
                          0.999, 1e-8, 1, _p(self.bf[k]))
        cqp_transpose_bf16(HID, HID, _p(self.bf["W2"]), _p(self.w2t))

    def forward(self, X, asset_off, count):
        torch = self.torch
        rows = X.shape[0]
        H1 = torch.empty(rows, HID, dtype=torch.bfloat16, device="cuda")
        H2 = torch.empty(rows, HID, dtype=torch.bfloat16, device="cuda")
        cqp_gemm_bf16(0, 0, rows, HID, FEAT, _p(X), FEAT, _p(self.bf["W1"]), HID, _p(H1), HID, _p(self.p["b1"]), 2)
        cqp_gemm_bf16(0, 1, rows, HID, HID, _p(H1), HID, _p(self.w2t), HID, _p(H2), HID, _p(self.p["b2"]), 2)
        score = torch.empty(rows, dtype=torch.float32, device="cuda")
        x0 = torch.empty(rows, dtype=torch.float32, device="cuda")
        pooled = torch.empty(count, HID, dtype=torch.float32, device="cuda")
        ydual = torch.empty(count, 2, dtype=torch.float32, device="cuda")
        cqp_ws_head_forward(count, _p(asset_off), _p(H2), _p(self.p["w3"]), _p(self.p["b3"]), _p(self.p["Wd"]),
                            _p(self.p["bd"]), _p(score), _p(x0), _p(pooled), _p(ydual))
        return dict(X=X, H1=H1, H2=H2, score=score, x0=x0, pooled=pooled, ydual=ydual, asset_off=asset_off,
                    count=count)

    def backward(self, f, xstar, ystar, lam=1.0):
        """Gradients of the mean (over instances) training loss into self.g; returns the loss."""
        torch = self.torch
        for t in self.g.values():
            t.zero_()
        rows, count = f["X"].shape[0], f["count"]
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        dscore = torch.empty(rows, dtype=torch.float32, device="cuda")
        dyd = torch.empty(count, 2, dtype=torch.float32, device="cuda")
        cqp_ws_loss(count, _p(f["asset_off"]), _p(f["x0"]), _p(xstar), _p(f["ydual"]), _p(ystar), lam, 1.0 / count,
                    _p(dscore), _p(dyd), _p(loss))
        dZ2 = torch.empty(rows, HID, dtype=torch.bfloat16, device="cuda")
        cqp_ws_head_backward(count, _p(f["asset_off"]), _p(f["H2"]), _p(self.p["w3"]), _p(self.p["Wd"]), _p(dscore),
                             _p(dyd), _p(f["pooled"]), _p(dZ2), _p(self.g["w3"]), _p(self.g["b3"]),
                             _p(self.g["Wd"]), _p(self.g["bd"]))
        cqp_relu_backward_bf16(rows, HID, _p(f["H2"]), _p(dZ2), _p(self.g["b2"]))
        split = max(1, min(256, rows // 2048))
        cqp_gemm_bf16(1, 0, HID, HID, rows, _p(f["H1"]), HID, _p(dZ2), HID, _p(self.g["W2"]), HID, None, 3, split)
        dH1 = torch.empty(rows, HID, dtype=torch.bfloat16, device="cuda")
        cqp_gemm_bf16(0, 1, rows, HID, HID, _p(dZ2), HID, _p(self.bf["W2"]), HID, _p(dH1), HID, None, 4)
        cqp_relu_backward_bf16(rows, HID, _p(f["H1"]), _p(dH1), _p(self.g["b1"]))
        cqp_gemm_bf16(1, 0, FEAT, HID, rows, _p(f["X"]), FEAT, _p(dH1), HID, _p(self.g["W1"]), HID, None, 3, split)
        # the intermediate derivatives stay available to the caller (layer-by-layer checks)
        f.update(dscore=dscore, dyd=dyd, dZ2=dZ2, dZ1=dH1)
        return loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        for k in PARAMS:
            cqp_adam_step(self.p[k].numel(), _p(self.p[k]), _p(self.g[k]), _p(self.m[k]), _p(self.v[k]), lr, beta1,
                          beta2, eps, self.step, _p(self.bf.get(k)))
        cqp_transpose_bf16(HID, HID, _p(self.bf["W2"]), _p(self.w2t))

    def start(self, dev: BatchDevice, X=None, dual_mode: int = 1):
        """(x0, y0) of the batch (FP64 device tensors) from the network.  dual_mode: 0 primal
        start only (y0 = 0), 1 budget and risk duals, 2 the whole dual from lambda = y_t / t."""
        torch = self.torch
        X = dev.features() if X is None else X
        f = self.forward(X, dev.asset_off, dev.count)
        x0 = torch.zeros(dev.n, dtype=torch.float64, device="cuda")
        y0 = torch.zeros(dev.m, dtype=torch.float64, device="cuda")
        cqp_ws_start(dev.count, _p(dev.x_off), _p(dev.row_off), _p(dev.n_assets), _p(dev.asset_off), _p(dev.rank),
                     _p(dev.q), _p(dev.R), dev.ldr, _p(dev.b), _p(f["x0"]), _p(f["ydual"]), YB_SCALE, dual_mode,
                     _p(x0), _p(y0))
        return x0, y0


class TrainingSet:
    """Features and targets of solved batches, resident on the device."""

    def __init__(self):
        self.parts = []

    def add(self, batch, x, y):
        import torch
        dev = BatchDevice(batch)
        xs, ys = targets(batch, np.asarray(x), np.asarray(y))
        self.parts.append(dict(X=dev.features(), off=dev.asset_off_h, xs=torch.from_numpy(xs).cuda(),
                               ys=torch.from_numpy(ys).cuda(), count=dev.count))

    def minibatch(self, rng, instances):
        import torch
        part = self.parts[int(rng.integers(len(self.parts)))]
        cnt = min(instances, part["count"])
        i0 = int(rng.integers(0, part["count"] - cnt + 1))
        off = part["off"]
        r0, r1 = int(off[i0]), int(off[i0 + cnt])
        aoff = torch.from_numpy((off[i0:i0 + cnt + 1] - r0).astype(np.int64)).cuda()
        return part["X"][r0:r1], aoff, cnt, part["xs"][r0:r1], part["ys"][i0:i0 + cnt]


def train(net: WarmStartNet, data: TrainingSet, steps: int, instances: int = 256, lr: float = 1e-3,
          lam: float = 1.0, seed: int = 0, log_every: int = 0):
    rng = np.random.default_rng(seed)
    hist = []
    for s in range(steps):
        X, aoff, cnt, xs, ys = data.minibatch(rng, instances)
        f = net.forward(X, aoff, cnt)
        loss = net.backward(f, xs, ys, lam)
        net.adam(lr)
        if log_every and (s % log_every == 0 or s == steps - 1):
            hist.append((s, float(loss.item()) / cnt))
    return hist


def solve_batch(batch, net: WarmStartNet | None = None, dual_mode: int = 1, fallback: bool = True, **opts):
    """Batched solve of a portfolio batch, from the network's start when `net` is given,
    else from zero.  Returns (x, y, per-instance results, summary).

    Plain cold-start PDHG stays the fallback of the learned start: with `fallback`, every
    instance whose warm-started solve ends unconverged (iteration or time limit, numerical
    error) is solved again from zero, in one more batched launch in which the converged
    instances start from their own solution (they stop at the first check).  The summary's
    "fallback" entry counts those instances."""
    dbatch = to_device(batch)
    s = BatchSolver(dbatch, device=True, **opts)
    try:
        if net is None:
            return s.solve(out_device=True)
        x0, y0 = net.start(BatchDevice(dbatch), dual_mode=dual_mode)
        x, y, per, res = s.solve(x0=x0, y0=y0, out_device=True)
        bad = [i for i, r in enumerate(per) if r["rc"] != 0]
        res["fallback"] = len(bad)
        if not bad or not fallback:
            return x, y, per, res
        xo, ro = dbatch["x_off"], dbatch["row_off"]
        xs, ys = x.clone(), y.clone()
        for i in bad:
            xs[int(xo[i]):int(xo[i + 1])] = 0.0
            ys[int(ro[i]):int(ro[i + 1])] = 0.0
        x2, y2, per2, res2 = s.solve(x0=xs, y0=ys, out_device=True)
        for i in bad:
            x[int(xo[i]):int(xo[i + 1])] = x2[int(xo[i]):int(xo[i + 1])]
            y[int(ro[i]):int(ro[i + 1])] = y2[int(ro[i]):int(ro[i + 1])]
            per[i] = per2[i]
        res["rc"] = max((r["rc"] for r in per), key=lambda v: (v != 0, abs(v)))
        res["kernel_ms"] += res2["kernel_ms"]
        res["fallback_kernel_ms"] = res2["kernel_ms"]
        return x, y, per, res
    finally:
        s.close()
