"""GPU tests of the learned warm start (include/cqp_mlp.h).

* the BF16 tensor-core GEMM against the exact product of the same BF16 values,
  for every transpose combination and epilogue, at ragged sizes;
* features, forward pass and gradients of the network against the FP64 oracle
  (oracle/mlp.py) evaluated on the same BF16-rounded weights and inputs;
* what training buys: on held-out portfolio batches the warm-started batched
  solve needs fewer iterations than the cold start and still reaches rel-KKT
  <= 1e-4 on every instance (the solver's own KKT test decides).
"""
import numpy as np
import pytest

import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_09159_gb300 as g
    g.build()
    g.lib()
    return g


def _bf16(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("ta", [0, 1])
@pytest.mark.parametrize("tb", [0, 1])
@pytest.mark.parametrize("epi", [0, 1, 2, 3, 4])
def test_gemm_bf16(gpu, ta, tb, epi):
    import torch
    rng = np.random.default_rng(10 + 4 * ta + 2 * tb + 16 * epi)
    M, N, K = 300, 200, 70 if epi != 3 else 1100
    A = rng.normal(size=(K, M) if ta else (M, K))
    B = rng.normal(size=(N, K) if tb else (K, N))
    At, Bt = _bf16(torch, A), _bf16(torch, B)
    Ab = At.float().cpu().numpy().astype(np.float64)
    Bb = Bt.float().cpu().numpy().astype(np.float64)
    ref = (Ab.T if ta else Ab) @ (Bb.T if tb else Bb)
    bias = rng.normal(size=N).astype(np.float32)
    bt = torch.from_numpy(bias).cuda()
    if epi in (2, 4):
        C = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    else:
        C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
        if epi == 3:
            C.fill_(0.5)
    gpu.cqp_gemm_bf16(ta, tb, M, N, K, At.data_ptr(), A.shape[1], Bt.data_ptr(), B.shape[1], C.data_ptr(), N,
                      bt.data_ptr() if epi in (1, 2) else None, epi, 7 if epi == 3 else 1)
    got = C.float().cpu().numpy().astype(np.float64)
    if epi in (1, 2):
        ref = ref + bias
    if epi == 2:
        ref = np.maximum(ref, 0.0)
    if epi == 3:
        ref = ref + 0.5
    bound = (np.abs(Ab.T if ta else Ab) @ np.abs(Bb.T if tb else Bb)) + 1.0
    tol = 2.0 ** -8 if epi in (2, 4) else 1e-5
    assert np.all(np.abs(got - ref) <= tol * bound), np.abs(got - ref).max()


def _net_params_numpy(net):
    import torch
    p = {k: v.double().cpu().numpy().copy() for k, v in net.p.items()}
    for k in ("W1", "W2"):
        p[k] = net.bf[k].float().cpu().numpy().astype(np.float64)   # the GEMMs use the BF16 copies
    return p


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_forward_and_gradients_match_oracle(gpu):
    import torch
    from oracle import mlp as M
    from paper_2608_09159_gb300 import warmstart as W
    b = I.portfolio_batch(count=6, n_range=(20, 50), k_range=(3, 8), seed=4242)
    dev = W.BatchDevice(b)
    X = dev.features()
    Xo = M.features(b, b["n_factors"])
    Xg = X.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Xg - Xo) <= 2.0 ** -8 * np.abs(Xo) + 1e-30)
    net = W.WarmStartNet(seed=5)
    rng = np.random.default_rng(6)
    # a non-trivial dual head and score layer
    net.p["Wd"].copy_(torch.from_numpy(rng.normal(size=(W.HID, 2)).astype(np.float32) * 0.05))
    net.p["w3"].copy_(torch.from_numpy(rng.normal(size=W.HID).astype(np.float32) * 0.05))
    off = dev.asset_off_h
    f = net.forward(X, dev.asset_off, dev.count)
    p = _net_params_numpy(net)
    fo = M.forward(p, Xg, off)
    assert _relerr(f["x0"].double().cpu().numpy(), fo["x0"]) <= 2e-2
    assert _relerr(f["ydual"].double().cpu().numpy(), fo["yd"]) <= 2e-2
    xs = np.concatenate([rng.dirichlet(np.ones(int(n))) for n in b["n_assets"]]).astype(np.float32)
    ys = rng.normal(size=(dev.count, 2)).astype(np.float32)
    loss = net.backward(f, torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda(), lam=1.0)
    go = M.backward(p, Xg, fo, xs.astype(np.float64), ys.astype(np.float64), off, 1.0)
    assert abs(loss.item() - M.loss(fo, xs, ys, off, 1.0)) <= 2e-2 * abs(M.loss(fo, xs, ys, off, 1.0))
    for k in W.PARAMS:
        gk = net.g[k].double().cpu().numpy() * dev.count          # the GPU gradient is of the mean loss
        if k == "b3":
            # a common shift of the scores leaves every softmax unchanged: the exact gradient is 0
            assert abs(gk[0]) <= 1e-4 * np.abs(go["w3"]).max(), gk
            continue
        assert _relerr(gk.reshape(go[k].shape), go[k]) <= 6e-2, k


def test_trained_start_needs_fewer_iterations(gpu):
    from paper_2608_09159_gb300 import warmstart as W
    opts = dict(precision=0, tol=1e-4, max_iter=100000, time_limit_s=120.0)
    data = W.TrainingSet()
    for seed in (501, 502):
        tb = I.portfolio_batch(count=600, n_range=(20, 60), k_range=(3, 8), seed=seed)
        x, y, per, res = W.solve_batch(tb, None, **opts)
        assert res["rc"] == 0
        data.add(tb, x.cpu().numpy(), y.cpu().numpy())
    net = W.WarmStartNet(seed=1)
    hist = W.train(net, data, steps=400, instances=64, lr=1e-3, log_every=100)
    assert hist[-1][1] < hist[0][1]
    test = I.portfolio_batch(count=200, n_range=(20, 60), k_range=(3, 8), seed=599)
    _, _, cold, rc = W.solve_batch(test, None, **opts)
    ic = np.mean([r["iters"] for r in cold])
    assert rc["rc"] == 0
    for mode in (0, 1):          # primal start only; primal start plus the budget and risk duals
        _, _, warm, rw = W.solve_batch(test, net, dual_mode=mode, **opts)
        assert rw["rc"] == 0
        assert max(r["kkt"]["rel_kkt"] for r in warm) <= 1e-4
        iw = np.mean([r["iters"] for r in warm])
        print("dual_mode %d: mean iterations cold %.1f warm %.1f" % (mode, ic, iw))
        assert iw < 0.95 * ic
