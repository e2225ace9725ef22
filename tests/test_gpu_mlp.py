"""GPU tests of the learned warm start (include/cqp_mlp.h).

* the BF16 tensor-core GEMM against the exact product of the same BF16 values,
  for every transpose combination and epilogue, at ragged sizes;
* features, forward pass and gradients of the network against the FP64 oracle
  (oracle/mlp.py), layer by layer and element by element: each layer's reference takes the
  same BF16 weights and the GPU's own BF16-rounded input of that layer, and the bound is one
  BF16 rounding of the output plus the FP32 accumulation error;
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


@pytest.mark.parametrize("shape", [(1, 256, 64), (77, 512, 192), (128, 256, 64), (300, 512, 128), (1000, 256, 576),
                                   (4100, 768, 512), (40000, 512, 256)])
@pytest.mark.parametrize("epi", [0, 1, 2, 4])
def test_gemm_tensor_memory_path(gpu, shape, epi):
    """C = A B' with A (M x K) and B (N x K) row-major: the form that runs on tcgen05.mma with
    the accumulator in tensor memory.  A single row and 77 rows (one partial tile: the tensor
    copies fill rows past M with zeros and the tiled stores clip them), one tile (128 x 256 x
    64), ragged row tiles (M = 300,
    1000, 4100), several K slices through the four-stage ring (K = 576: nine slices, the ring
    wraps twice), several column tiles, and more tiles than SMs (M = 40,000: 626 tiles, so each
    persistent block alternates its two tensor-memory accumulators); compared with the exact
    product of the same BF16 values, and the launch counter shows the tensor-memory kernel ran."""
    import torch
    M, N, K = shape
    rng = np.random.default_rng(M + N + K + epi)
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(N, K))
    At, Bt = _bf16(torch, A), _bf16(torch, B)
    Ab = At.float().cpu().numpy().astype(np.float64)
    Bb = Bt.float().cpu().numpy().astype(np.float64)
    ref = Ab @ Bb.T
    bias = rng.normal(size=N).astype(np.float32)
    bt = torch.from_numpy(bias).cuda()
    if epi in (2, 4):
        C = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
    else:
        C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    before = gpu.lib().cqp_gemm_tc_launches()
    gpu.cqp_gemm_bf16(0, 1, M, N, K, At.data_ptr(), K, Bt.data_ptr(), K, C.data_ptr(), N,
                      bt.data_ptr() if epi in (1, 2) else None, epi, 1)
    gpu.cqp_gemm_check()
    assert gpu.lib().cqp_gemm_tc_launches() == before + 1
    got = C.float().cpu().numpy().astype(np.float64)
    if epi in (1, 2):
        ref = ref + bias
    if epi == 2:
        ref = np.maximum(ref, 0.0)
    bound = np.abs(Ab) @ np.abs(Bb.T) + 1.0
    tol = 2.0 ** -8 if epi in (2, 4) else 1e-5
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= tol * bound), np.abs(got - ref).max()


def test_gemm_tensor_memory_path_strided(gpu):
    """Leading dimensions above the row lengths (lda = K + 64, ldb = K + 8, ldc = N + 256): the
    tensor maps' row strides and the epilogue's stores honour them, and the padding of C is
    left untouched."""
    import torch
    M, N, K = 260, 256, 128
    rng = np.random.default_rng(77)
    A = _bf16(torch, rng.normal(size=(M, K + 64)))
    B = _bf16(torch, rng.normal(size=(N, K + 8)))
    C = torch.full((M, N + 256), 7.0, dtype=torch.float32, device="cuda")
    before = gpu.lib().cqp_gemm_tc_launches()
    gpu.cqp_gemm_bf16(0, 1, M, N, K, A.data_ptr(), K + 64, B.data_ptr(), K + 8, C.data_ptr(), N + 256, None, 0, 1)
    gpu.cqp_gemm_check()
    assert gpu.lib().cqp_gemm_tc_launches() == before + 1
    Ab = _np(A)[:, :K]
    Bb = _np(B)[:, :K]
    got = C.cpu().numpy().astype(np.float64)
    ref = Ab @ Bb.T
    assert np.all(np.abs(got[:, :N] - ref) <= 1e-5 * (np.abs(Ab) @ np.abs(Bb.T) + 1.0))
    assert np.all(got[:, N:] == 7.0)
    # a bias pointer off the 16-byte grid takes the warp-level kernel, with the same result
    bias = torch.from_numpy(rng.normal(size=N + 1).astype(np.float32)).cuda()
    C2 = torch.empty(M, N, dtype=torch.float32, device="cuda")
    before = gpu.lib().cqp_gemm_tc_launches()
    gpu.cqp_gemm_bf16(0, 1, M, N, K, A.data_ptr(), K + 64, B.data_ptr(), K + 8, C2.data_ptr(), N,
                      bias[1:].data_ptr(), 1, 1)
    assert gpu.lib().cqp_gemm_tc_launches() == before
    ref1 = ref + bias[1:].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(C2.cpu().numpy() - ref1) <= 1e-5 * (np.abs(Ab) @ np.abs(Bb.T) + 1.0))


def _net_params_numpy(net):
    p = {k: v.double().cpu().numpy().copy() for k, v in net.p.items()}
    for k in ("W1", "W2"):
        p[k] = net.bf[k].float().cpu().numpy().astype(np.float64)   # the GEMMs use the BF16 copies
    return p


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


U32 = 2.0 ** -24        # FP32 unit roundoff
BF16 = 2.0 ** -8        # one BF16 rounding (round to nearest: 2^-9 relative), with margin


def _check(name, got, ref, terms, k, bf16_out):
    """Elementwise: |got - ref| <= (BF16 rounding of ref if the kernel writes BF16) + k u32 * terms,
    with terms the sum of |products| of each entry's FP32 accumulation of length k."""
    bound = (BF16 * np.abs(ref) if bf16_out else 0.0) + 2.0 * k * U32 * terms + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= bound), (name, float(err.max()), float((err / bound).max()))


def test_forward_and_gradients_match_oracle_elementwise(gpu):
    """Every layer of the BF16 network, forward and backward, against oracle/mlp.py evaluated in FP64
    on the same BF16 weights and on the GPU's own (BF16-rounded) inputs of that layer, element by
    element, with a bound from one BF16 rounding of the output and the FP32 accumulation."""
    import torch
    from oracle import mlp as M
    from paper_2608_09159_gb300 import warmstart as W
    b = I.portfolio_batch(count=6, n_range=(20, 50), k_range=(3, 8), seed=4242)
    dev = W.BatchDevice(b)
    X = dev.features()
    Xo = M.features(b, b["n_factors"])
    Xg = _np(X)
    assert np.all(np.abs(Xg - Xo) <= BF16 * np.abs(Xo) + 1e-30)
    net = W.WarmStartNet(seed=5)
    rng = np.random.default_rng(6)
    # a non-trivial dual head and score layer
    net.p["Wd"].copy_(torch.from_numpy(rng.normal(size=(W.HID, 2)).astype(np.float32) * 0.05))
    net.p["w3"].copy_(torch.from_numpy(rng.normal(size=W.HID).astype(np.float32) * 0.05))
    net.p["b1"].copy_(torch.from_numpy(rng.normal(size=W.HID).astype(np.float32) * 0.05))
    net.p["b2"].copy_(torch.from_numpy(rng.normal(size=W.HID).astype(np.float32) * 0.05))
    off = dev.asset_off_h
    count, rows = dev.count, Xg.shape[0]
    f = net.forward(X, dev.asset_off, count)
    p = _net_params_numpy(net)
    A = np.abs
    # layer 1 from the features, layer 2 from the GPU's BF16 H1, head from the GPU's BF16 H2
    _, H1r = M.layer(Xg, p["W1"], p["b1"])
    H1g = _np(f["H1"])
    _check("H1", H1g, H1r, A(Xg) @ A(p["W1"]) + A(p["b1"]), Xg.shape[1] + 1, True)
    _, H2r = M.layer(H1g, p["W2"], p["b2"])
    H2g = _np(f["H2"])
    _check("H2", H2g, H2r, A(H1g) @ A(p["W2"]) + A(p["b2"]), W.HID + 1, True)
    hr = M.head_forward(p, H2g, off)
    sg = _np(f["score"])
    _check("score", sg, hr["s"], A(H2g) @ A(p["w3"]) + A(p["b3"][0]), W.HID + 1, False)
    # softmax of the GPU's own scores, and the pooled mean / dual head of its H2
    hs = M.head_forward(p, H2g, off)
    x0g = _np(f["x0"])
    xs_ref = np.empty_like(sg)
    for i in range(count):
        z = np.exp(sg[off[i]:off[i + 1]] - sg[off[i]:off[i + 1]].max())
        xs_ref[off[i]:off[i + 1]] = z / z.sum()
    assert np.all(np.abs(x0g - xs_ref) <= 256 * U32 * xs_ref + 1e-12)
    pg = _np(f["pooled"])
    assert np.all(np.abs(pg - hs["pooled"]) <= 2 * 64 * U32 * (A(H2g).max() + 1e-30))
    _check("ydual", _np(f["ydual"]), pg @ p["Wd"] + p["bd"], A(pg) @ A(p["Wd"]) + A(p["bd"]), W.HID + 1, False)
    # backward: loss gradients of the mean loss (scale 1/count) from the GPU's forward values
    xs = np.concatenate([rng.dirichlet(np.ones(int(n))) for n in b["n_assets"]]).astype(np.float32)
    ys = rng.normal(size=(count, 2)).astype(np.float32)
    loss = net.backward(f, torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda(), lam=1.0)
    fg = dict(s=sg, x0=x0g, pooled=pg, yd=_np(f["ydual"]), H2=H2g)
    ds, dyd, _, gh = M.head_backward(p, fg, xs.astype(np.float64), ys.astype(np.float64), off, 1.0)
    assert abs(loss.item() - M.loss(fg, xs, ys, off, 1.0)) <= 1e-5 * M.loss(fg, xs, ys, off, 1.0)
    dsg, dydg = _np(f["dscore"]), _np(f["dyd"])
    big = 1.0 + max(A(ds).max(), A(dyd).max()) / count
    assert np.all(A(dsg - ds / count) <= 256 * U32 * big), float(A(dsg - ds / count).max())
    assert np.all(A(dydg - dyd / count) <= 16 * U32 * big)
    # head parameter gradients from the GPU's own dscore and dydual
    gw3r, gb3r, _ = M.layer_backward(H2g, dsg[:, None])
    gWdr, gbdr, _ = M.layer_backward(pg, dydg)
    for k, ref, terms, K in (("w3", gw3r[:, 0], A(H2g).T @ A(dsg), rows), ("b3", gb3r, A(dsg).sum(keepdims=True), rows),
                             ("Wd", gWdr, A(pg).T @ A(dydg), count), ("bd", gbdr, A(dydg).sum(axis=0), count)):
        _check("g" + k, _np(net.g[k]).reshape(ref.shape), ref, terms, K + 8, False)
    assert np.all(A(gw3r[:, 0] - gh["w3"] / count) <= 1e-4 * (A(gh["w3"]).max() / count + 1e-30))
    # the masked dZ2 from the GPU's ds, dyd; layer-2 gradients and dZ1 from the GPU's BF16 dZ2
    dZ2r = M.head_input_grad(p, dsg, dydg, off) * (H2g > 0)
    dZ2g = _np(f["dZ2"])
    _check("dZ2", dZ2g, dZ2r, (A(dsg)[:, None] * A(p["w3"])[None, :] + A(dydg @ p["Wd"].T).max()) * (H2g > 0), 4, True)
    gW2r, gb2r, dZ1r = M.layer_backward(H1g, dZ2g, p["W2"], H1g > 0)
    _check("gW2", _np(net.g["W2"]), gW2r, A(H1g).T @ A(dZ2g), rows, False)
    _check("gb2", _np(net.g["b2"]), gb2r, A(dZ2g).sum(axis=0), rows, False)
    dZ1g = _np(f["dZ1"])
    _check("dZ1", dZ1g, dZ1r, (A(dZ2g) @ A(p["W2"]).T) * (H1g > 0), W.HID, True)
    gW1r, gb1r, _ = M.layer_backward(Xg, dZ1g)
    _check("gW1", _np(net.g["W1"]), gW1r, A(Xg).T @ A(dZ1g), rows, False)
    _check("gb1", _np(net.g["b1"]), gb1r, A(dZ1g).sum(axis=0), rows, False)


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


def test_unconverged_warm_start_falls_back_to_cold_start(gpu):
    """A network whose dual head is far off (bias 1e4) leaves its warm-started instances unconverged
    within the iteration cap; solve_batch then solves them again from zero, the plain method."""
    import torch
    from paper_2608_09159_gb300 import warmstart as W
    test = I.portfolio_batch(count=40, n_range=(20, 60), k_range=(3, 8), seed=598)
    _, _, cold, rc = W.solve_batch(test, None, precision=0, tol=1e-4, max_iter=100000, time_limit_s=120.0)
    assert rc["rc"] == 0
    cap = max(r["iters"] for r in cold)
    net = W.WarmStartNet(seed=3)
    net.p["bd"].copy_(torch.tensor([1e4, -1e4], dtype=torch.float32))
    opts = dict(precision=0, tol=1e-4, max_iter=cap, time_limit_s=120.0)
    _, _, warm, rw = W.solve_batch(test, net, dual_mode=1, fallback=False, **opts)
    failed = [i for i, r in enumerate(warm) if r["rc"] != 0]
    assert rw["fallback"] == len(failed) > 0
    x, y, per, rf = W.solve_batch(test, net, dual_mode=1, **opts)
    assert rf["fallback"] == len(failed)
    assert all(r["rc"] == 0 for r in per) and rf["rc"] == 0
    for i in failed:                      # the fallback instances are the cold solves
        assert per[i]["iters"] == cold[i]["iters"]
        assert per[i]["kkt"]["rel_kkt"] <= 1e-4
