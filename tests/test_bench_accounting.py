"""Host checks of bench.py's byte accounting (the numerator of every roofline fraction it prints):
the per-unit figures of the measurement section, written out by hand for a small case, and the
BF16 variant's value bytes."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_for_tests", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_algorithmic_bytes_by_hand():
    b = _bench()
    n, m, nnz, iters, inner, k, pnnz = 1000, 400, 7000, 128, 300, 5, 2000
    # per outer iteration: A'y (values + indices, n + 1 row pointers, gather y once, write v) and
    # A x (values + indices, m + 1 row pointers, gather x once, write m); per inner step: R and R'
    # (2 k n), P (values + indices + n + 1 row pointers) and eight n-vectors; a check every 64
    # iterations (plus the last) repeats the two products
    per_iter = (nnz * 8 + (n + 1) * 4 + m * 4 + n * 4) + (nnz * 8 + (m + 1) * 4 + n * 4 + m * 4)
    per_inner = 2 * k * n * 4 + (pnnz * 8 + (n + 1) * 4) + 8 * n * 4
    checks = iters // 64 + 1
    want = iters * per_iter + inner * per_inner + checks * per_iter
    assert b.algorithmic_bytes(n, m, nnz, iters, inner, k, pnnz) == want


def test_bf16_values_count_two_bytes():
    b = _bench()
    n, m, nnz, iters, inner, pnnz = 2000, 500, 10000, 64, 100, 4000
    f32 = b.algorithmic_bytes(n, m, nnz, iters, inner, 0, pnnz)
    bf16 = b.algorithmic_bytes(n, m, nnz, iters, inner, 0, pnnz, vsize=2)
    checks = iters // 64 + 1
    # two bytes less per stored value of A and A' per product, and of P per inner step
    assert f32 - bf16 == 2 * (2 * nnz) * (iters + checks) + 2 * pnnz * inner


def test_source_hash_covers_the_solver_kernel_sources():
    b = _bench()
    csrc = os.path.join(ROOT, "paper_2608_09159_gb300", "csrc")
    for f in b.SOLVER_SOURCES:
        assert os.path.exists(os.path.join(csrc, f)), f
    assert "solver_grid_f32.cu" in b.SOLVER_SOURCES   # the translation unit of pdhg_grid_kernel<float>
    h = b._source_hash()
    assert len(h) == 16 and h == b._source_hash()
