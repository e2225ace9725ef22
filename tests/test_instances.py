"""Input generators: Philox-4x32-10 known answers and instance structure."""
import numpy as np

import instances as I


def test_philox_known_answers():
    # Known-answer vectors published with the Philox definition (Salmon et al., SC 2011; Random123 KAT file)
    z = I.philox4x32_10(np.zeros((1, 4), np.uint32), np.zeros(2, np.uint32))[0]
    assert [int(v) for v in z] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    f = I.philox4x32_10(np.full((1, 4), 0xFFFFFFFF, np.uint32), np.full(2, 0xFFFFFFFF, np.uint32))[0]
    assert [int(v) for v in f] == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    pi = I.philox4x32_10(np.array([[0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], np.uint32),
                         np.array([0xA4093822, 0x299F31D0], np.uint32))[0]
    assert [int(v) for v in pi] == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_stream_reproducible_and_distributions():
    a = I.Stream(7, 3).uniform(50000)
    b = I.Stream(7, 3).uniform(50000)
    assert np.array_equal(a, b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.01
    z = I.Stream(8, 0).normal(100000)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


def _check_structure(inst):
    n, m = inst["n"], inst["m"]
    assert inst["a_rowptr"].size == m + 1 and inst["a_rowptr"][0] == 0
    assert inst["a_colind"].min() >= 0 and inst["a_colind"].max() < n
    # blocks partition 0..n-1 contiguously
    s, d = inst["blk_start"], inst["blk_dim"]
    assert s[0] == 0 and np.all(s[1:] == s[:-1] + d[:-1]) and s[-1] + d[-1] == n
    assert inst["c"].size == n and inst["b"].size == m


def test_small_configs_structure_and_feasibility():
    for k in (1, 2, 3):
        inst = I.small_config(k)
        _check_structure(inst)
        if "x_feasible" in inst:
            x0 = inst["x_feasible"]
            assert np.allclose(I.csr_matvec(inst["a_rowptr"], inst["a_colind"], inst["a_val"], x0), inst["b"])


def test_fisher_rows():
    # eq. fisher-conic as counted after it: e + 4n stored coordinates and m + n equations with the
    # middle coordinates fixed by the block type; one more row per buyer in the explicit-row form
    inst = I.small_config(3)
    f = inst["fisher"]
    nb, ng = f["n_buyers"], f["n_goods"]
    assert inst["m"] == ng + nb
    assert inst["n"] == f["edges"] + 4 * nb
    assert set(inst["blk_type"][1:]) <= {I.CONE_EXP1, I.CONE_POW1}
    # every supply row and utility row is non-empty
    assert np.all(np.diff(inst["a_rowptr"]) > 0)
    rw = I.fisher_market(n_buyers=200, n_goods=40, density=0.1, seed=2003, fixed_middle=False)
    assert rw["m"] == ng + 2 * nb and rw["n"] == inst["n"]
    assert set(rw["blk_type"][1:]) <= {I.CONE_EXP, I.CONE_POW}
    assert np.all(np.diff(rw["a_rowptr"]) > 0)


def test_portfolio_batch_structure():
    # members cut out of the batch reproduce the batch; every row and entry stays inside
    # its instance; the equal-weight portfolio is feasible and on the risk bound
    b = I.portfolio_batch(count=5, n_range=(6, 12), k_range=(2, 4), seed=77)
    assert b["x_off"][-1] == b["n"] and b["row_off"][-1] == b["m"]
    rp, ci = b["a_rowptr"], b["a_colind"]
    for i in range(b["batch_count"]):
        x0, x1 = b["x_off"][i], b["x_off"][i + 1]
        for r in range(b["row_off"][i], b["row_off"][i + 1]):
            cols = ci[rp[r]:rp[r + 1]]
            assert cols.min() >= x0 and cols.max() < x1
        m = I.batch_member(b, i)
        n_as, k = int(b["n_assets"][i]), int(b["n_factors"][i])
        assert m["n"] == 2 * n_as + k + 1 and m["m"] == n_as + k + 2
        F = m["q_R"][:k, :n_as].T
        D = m["q_diag"][:n_as]
        xe = np.full(n_as, 1.0 / n_as)
        z = np.concatenate([xe, F.T @ xe, np.sqrt(D) * xe, [m["b"][-1]]])
        assert np.allclose(I.csr_matvec(m["a_rowptr"], m["a_colind"], m["a_val"], z), m["b"], atol=1e-12)
        assert abs(np.linalg.norm(z[n_as:-1]) - z[-1]) <= 1e-12
        assert list(m["blk_type"]) == [I.CONE_NONNEG, I.CONE_SOC]


def test_round_bf16_is_round_to_nearest_even():
    # against torch's FP32 -> BF16 conversion (round to nearest, ties to even) on random values,
    # exact ties, values next to a power of two and signed zeros
    import torch
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-30, 30, size=20000),
                        [0.0, -0.0, 1.0, -1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, 2.0 - 2.0 ** -9]])
    got = I.round_bf16(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(got, ref)
    assert np.array_equal(np.signbit(got), np.signbit(ref))
    # the ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and goes to the even 1; 1 + 3 2^-8 goes up
    assert got[-4] == 1.0 and got[-3] == 1.0 + 2.0 ** -6
    # the bit patterns reproduce the rounded values
    bits = I.bf16_bits(x).astype(np.uint32) << 16
    assert np.array_equal(bits.view(np.float32).astype(np.float64), got)


def test_bf16_rounding_and_positive_semidefiniteness_of_p():
    # BF16 storage of P (matrix_bf16 = 2) solves the problem with P rounded entrywise.  For the
    # large QP's P (a diagonal plus a weighted matching Laplacian: rows (i, j) hold d_i + w, -w) both
    # signs of a weight round alike, so every 2 x 2 block stays positive semidefinite; for the
    # sparse QP's P = M'M + 1e-2 I at full size the rounded matrix is indefinite
    inst = I.small_config(5)
    n = inst["n"]
    rp, ci, v = inst["p_rowptr"], inst["p_colind"], I.round_bf16(inst["p_val"])
    assert np.all(np.diff(rp) == 2)
    rows = np.repeat(np.arange(n), 2)
    diag = np.zeros(n)
    off = np.zeros(n)
    mate = np.full(n, -1)
    on = ci == rows
    diag[rows[on]] = v[on]
    off[rows[~on]] = v[~on]
    mate[rows[~on]] = ci[~on]
    assert np.all(mate >= 0) and np.all(mate[mate] == np.arange(n))
    assert np.all(off == off[mate])                                # symmetric after rounding
    assert np.all(diag >= 0) and np.all(diag * diag[mate] >= off * off)
    full = I.sparse_qp_nonneg()
    m = full["n"]
    P = np.zeros((m, m))
    r = np.repeat(np.arange(m), np.diff(full["p_rowptr"]))
    P[r, full["p_colind"]] = I.round_bf16(full["p_val"])
    assert np.linalg.eigvalsh(P).min() < 0.0
