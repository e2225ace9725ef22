"""GPU parity of the kernel-level entry points against the FP64 oracle.

SpMV and cone projections are called through the C ABI (cqp_spmv,
cqp_project) on device buffers and compared element by element with the
oracle on the same seeded inputs.  Tolerances: 1e-12 relative in FP64 and
1e-5 relative in FP32 (scaled by the row's |A||x| for products and by the
input's magnitude for projections).
"""
import numpy as np
import pytest

import _cones as G

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


def _csr_random(rng, m, n, density, long_rows=0):
    A = (rng.uniform(size=(m, n)) < density) * rng.normal(size=(m, n))
    A[rng.integers(0, m, size=max(1, m // 20))] = 0.0            # empty rows
    for r in rng.integers(0, m, size=long_rows):
        A[r] = rng.normal(size=n)                                   # dense rows
    rows, cols = np.nonzero(A)
    rp = np.zeros(m + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return A, np.cumsum(rp), cols, A[rows, cols]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("tpr", [-1, 0, 1, 2, 4, 8, 16, 32])
def test_spmv_parity(gpu, orc, rng, precision, tpr):
    import torch
    m, n = 1537, 1203                                               # ragged tail over many tiles
    A, rp, ci, v = _csr_random(rng, m, n, 0.01, long_rows=3)
    x = rng.normal(size=n)
    dt = torch.float64 if precision else torch.float32
    vt = torch.tensor(v, dtype=dt, device="cuda")
    xt = torch.tensor(x, dtype=dt, device="cuda")
    yt = torch.zeros(m, dtype=dt, device="cuda")
    rpt = torch.tensor(rp, dtype=torch.int32, device="cuda")
    cit = torch.tensor(ci, dtype=torch.int32, device="cuda")
    gpu.cqp_spmv(precision, m, n, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(), xt.data_ptr(), yt.data_ptr(), tpr)
    # oracle on the values as the GPU sees them (rounded to the precision)
    vr, xr = vt.double().cpu().numpy(), xt.double().cpu().numpy()
    ref = orc.spmv(rp, ci, vr, xr)
    scale = orc.spmv(rp, ci, np.abs(vr), np.abs(xr)) + 1e-300
    err = np.abs(yt.double().cpu().numpy() - ref) / scale
    assert err.max() <= (1e-12 if precision else 1e-5)


def _blocks_sample(rng):
    blist = []
    for t, d in [(G.NONNEG, 7), (G.SOC, 5), (G.RSOC, 6), (G.EXP, 3), (G.POW, 3), (G.FREE, 4), (G.SOC, 2),
                 (G.RSOC, 3), (G.SOC, 200), (G.RSOC, 150), (G.NONNEG, 1), (G.EXP1, 3), (G.POW1, 3)]:
        blist.append((t, d, float(rng.uniform(0.15, 0.85)) if t in (G.POW, G.POW1) else 0.0))
    blist = blist * 40
    types = np.array([b[0] for b in blist], np.int32)
    dims = np.array([b[1] for b in blist], np.int64)
    alphas = np.array([b[2] for b in blist])
    starts = np.zeros_like(dims)
    starts[1:] = np.cumsum(dims)[:-1]
    return types, starts, dims, alphas


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("metric", [False, True])
def test_projection_parity(gpu, orc, rng, precision, metric):
    import torch
    types, starts, dims, alphas = _blocks_sample(rng)
    n = int(dims.sum())
    r = rng.normal(size=n) * np.repeat(10.0 ** rng.uniform(-2, 2, size=types.size), dims)
    mvec = np.exp(rng.normal(size=n) * 0.7) if metric else None
    dt = torch.float64 if precision else torch.float32
    rt = torch.tensor(r, dtype=dt, device="cuda")
    mt = None if mvec is None else torch.tensor(mvec, dtype=dt, device="cuda")
    out = torch.zeros(n, dtype=dt, device="cuda")
    dev = [torch.tensor(a, device="cuda") for a in (types, starts, dims, alphas)]
    K = gpu.Cones(types.size, *[a.data_ptr() for a in dev])
    gpu.cqp_project(precision, n, K, rt.data_ptr(), None if mt is None else mt.data_ptr(), out.data_ptr())
    got = out.double().cpu().numpy()
    rr = rt.double().cpu().numpy()
    mm = None if mt is None else mt.double().cpu().numpy()
    tol = 1e-12 if precision else 1e-5
    for t, s, d, a in zip(types, starts, dims, alphas):
        ref = orc.proj_block(int(t), rr[s:s + d], alpha=a, m=None if mm is None else mm[s:s + d])
        scale = 1.0 + np.abs(rr[s:s + d]).max()
        lim = tol * scale
        assert np.abs(got[s:s + d] - ref).max() <= lim, (int(t), int(d), rr[s:s + d][:6], got[s:s + d][:6], ref[:6])


def test_projection_edge_cases(gpu, orc):
    import torch
    # points in K, in -K*, on case boundaries, exp face, power r_z = 0, RSOC singular
    cases = [(G.SOC, [0.3, 0.4, 1.0]), (G.SOC, [0.3, 0.4, -1.0]), (G.SOC, [3.0, 4.0, 5.0]), (G.SOC, [0.0, 0.0, 0.0]),
             (G.EXP, [0.0, 1.0, 2.0]), (G.EXP, [1.0, -1.0, -3.0]), (G.EXP, [-1.0, -2.0, 3.0]),
             (G.EXP, [-0.985, 0.00136, -1.83]), (G.POW, [-1.0, 2.0, 0.0]), (G.POW, [1.0, 1.0, 1.0]),
             (G.RSOC, [1.0, 2.0, -2.0]), (G.RSOC, [0.0, 0.0, 1.0, -1.0]), (G.NONNEG, [-1.0, 0.0, 2.0]),
             # slices: inside, c0 <= 0, large r0, z0 = 0, x0 < 0 with z0 != 0, on the boundary
             (G.EXP1, [0.0, 5.0, 2.0]), (G.EXP1, [1.0, 0.0, -3.0]), (G.EXP1, [30.0, 1.0, 0.5]),
             (G.EXP1, [-40.0, 1.0, -1e-3]), (G.EXP1, [0.5, 1.0, np.exp(0.5)]),
             (G.POW1, [-1.0, 2.0, 0.0]), (G.POW1, [-2.0, 1.0, 0.3]), (G.POW1, [4.0, 1.0, 4.0 ** 0.4]),
             (G.POW1, [1e-3, 1.0, -5.0]), (G.POW1, [50.0, 0.0, 1e-4]),
             # slices far outside: e^{r0} overflowing the naive bracket, |t0| >> 1
             (G.EXP1, [108.9, 18.0, -62.6]), (G.EXP1, [300.0, 1.0, 1e10]), (G.EXP1, [-5.0, 1.0, -1e4]),
             (G.POW1, [-3.0, 1.0, 1e4]), (G.POW1, [0.5, 1.0, -1e3]), (G.POW1, [1e4, 1.0, 1e6])]
    for precision in (0, 1):
        dt = torch.float64 if precision else torch.float32
        for t, r in cases:
            r = np.array(r)
            d = r.size
            dev = [torch.tensor(a, device="cuda") for a in (np.array([t], np.int32), np.array([0], np.int64),
                                                           np.array([d], np.int64), np.array([0.4]))]
            K = gpu.Cones(1, *[a.data_ptr() for a in dev])
            rt = torch.tensor(r, dtype=dt, device="cuda")
            out = torch.zeros(d, dtype=dt, device="cuda")
            gpu.cqp_project(precision, d, K, rt.data_ptr(), None, out.data_ptr())
            ref = orc.proj_block(t, rt.double().cpu().numpy(), alpha=0.4)
            assert np.allclose(out.double().cpu().numpy(), ref, atol=(1e-12 if precision else 1e-6) * (1 + np.abs(r).max()))
