"""GPU parity of the general standard form (cqp_setup_general): row bounds
lo <= Ax <= hi and box blocks, against the oracle's pinned general form.

* a box-constrained QP equals its closed form clip(-c/q, lo, hi);
* QPs with equality, one-sided and two-sided rows over nonnegative, box and
  second-order-cone blocks reach rel-KKT <= 1e-4 as re-measured by the oracle and
  match the oracle's objective, in FP32 and FP64;
* the KKT entry point equals the oracle's KKT at arbitrary points;
* inverted or NaN bounds are rejected.
"""
import numpy as np
import pytest

import instances as I
from _parity import REL_KKT, TIGHT_TOL, obj_close

pytestmark = pytest.mark.gpu
BOX = 6


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_09159_gb300 as g
    g.build()
    g.lib()
    return g


def _inst(A, c, blocks, q=None, lo=None, hi=None, xlo=None, xhi=None):
    m, n = A.shape
    r, ci = np.nonzero(A)
    rp, cc, v = I._coo_to_csr(m, n, r, ci, A[r, ci])
    bt, bs, bd, ba = I.blocks_from_list(blocks)
    inst = I.make_instance("g", m, n, rp, cc, v, c, np.zeros(m), bt, bs, bd, ba, q_diag=q)
    inst["row_lo"], inst["row_hi"] = np.asarray(lo, float), np.asarray(hi, float)
    if xlo is not None:
        inst["x_lo"], inst["x_hi"] = np.asarray(xlo, float), np.asarray(xhi, float)
    return inst


def _mixed(seed, m=60, n=150):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, n)) * (rng.uniform(size=(m, n)) < 0.15)
    for i in range(m):
        if not A[i].any():
            A[i, rng.integers(n)] = 1.0
    nn, nsoc, nbox = 70, 30, n - 100
    x0 = np.concatenate([np.abs(rng.normal(size=nn)), np.zeros(nsoc), rng.uniform(-0.5, 0.5, nbox)])
    x0[nn:nn + nsoc - 1] = rng.normal(size=nsoc - 1) * 0.1
    x0[nn + nsoc - 1] = np.linalg.norm(x0[nn:nn + nsoc - 1]) + 0.5
    ax0 = A @ x0
    lo = ax0 - rng.uniform(0.1, 1.0, m)
    hi = ax0 + rng.uniform(0.1, 1.0, m)
    lo[:15] = hi[:15] = ax0[:15]
    lo[15:25] = -np.inf
    hi[25:35] = np.inf
    xlo = np.full(n, -np.inf)
    xhi = np.full(n, np.inf)
    xlo[100:], xhi[100:] = -1.0, 1.0
    xlo[100:105] = -np.inf
    c = rng.normal(size=n)
    q = rng.uniform(0.1, 1.0, n)
    return _inst(A, c, [(I.CONE_NONNEG, nn, 0.0), (I.CONE_SOC, nsoc, 0.0), (BOX, nbox, 0.0)], q=q, lo=lo, hi=hi,
                 xlo=xlo, xhi=xhi)


def test_box_qp_closed_form(gpu):
    rng = np.random.default_rng(21)
    n = 300
    q = rng.uniform(0.5, 2.0, n)
    c = rng.normal(size=n) * 2
    lo, hi = rng.uniform(-1.0, 0.0, n), rng.uniform(0.0, 1.0, n)
    lo[:20] = -np.inf
    hi[20:40] = np.inf
    A = np.zeros((1, n + 1))
    A[0, n] = 1.0
    inst = _inst(A, np.concatenate([c, [0.0]]), [(BOX, n, 0.0), (I.CONE_FREE, 1, 0.0)],
                 q=np.concatenate([q, [1.0]]), lo=[0.0], hi=[0.0],
                 xlo=np.concatenate([lo, [0.0]]), xhi=np.concatenate([hi, [0.0]]))
    s = gpu.Solver(inst, precision=1, tol=1e-9, max_iter=200000, time_limit_s=60.0)
    x, y, res = s.solve()
    s.close()
    assert res["rc"] == 0
    assert np.abs(x[:n] - np.clip(-c / q, lo, hi)).max() <= 1e-6


@pytest.mark.parametrize("precision", [1, 0])
def test_mixed_rows_and_blocks_match_oracle(gpu, orc, precision):
    inst = _mixed(22)
    s = gpu.Solver(inst, precision=precision, tol=1e-4, max_iter=200000, time_limit_s=120.0)
    x, y, res = s.solve()
    s.close()
    assert res["rc"] == 0, res
    rep = orc.kkt(inst, x, y)
    assert rep["rel_kkt"] <= REL_KKT, rep
    assert abs(rep["rel_kkt"] - res["kkt"]["rel_kkt"]) <= 1e-7 + 1e-3 * rep["rel_kkt"]
    xo, yo, info = orc.solve(inst, max_iter=1000000, tol=TIGHT_TOL)
    assert obj_close(rep["pobj"], info["kkt"]["pobj"]), (rep["pobj"], info["kkt"]["pobj"])


def test_kkt_entry_point_general(gpu, orc):
    inst = _mixed(23)
    s = gpu.Solver(inst, precision=1)
    rng = np.random.default_rng(5)
    for _ in range(3):
        x, y = rng.normal(size=inst["n"]), rng.normal(size=inst["m"])
        rep, ref = s.kkt(x, y), orc.kkt(inst, x, y)
        for key in ("eps_p", "eps_d", "eps_g", "pobj", "dobj"):
            assert abs(rep[key] - ref[key]) <= 1e-10 * (1 + abs(ref[key])), key
    s.close()


def test_invalid_bounds(gpu):
    inst = _mixed(24)
    bad = dict(inst)
    bad["row_lo"] = inst["row_lo"].copy()
    bad["row_lo"][40] = inst["row_hi"][40] + 1.0
    with pytest.raises(gpu.CQPError) as e:
        gpu.Solver(bad)
    assert e.value.code == -1
    bad = dict(inst)
    bad["x_hi"] = inst["x_hi"].copy()
    bad["x_hi"][120] = np.nan
    with pytest.raises(gpu.CQPError) as e:
        gpu.Solver(bad)
    assert e.value.code == -1
