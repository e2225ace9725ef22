"""The OpenMP build of the oracle (liboracle_omp.so) repeats the single-threaded one exactly.

bench.py times the CPU baseline with both builds (one core and all host cores).  Its
parallel loops touch independent rows, coordinates and cone blocks, and every long
sum is taken in fixed chunks added in index order, so the iterates must be
bit-identical to the single-threaded build for any thread count.
"""
import numpy as np
import pytest

import instances as I


@pytest.mark.parametrize("k", [1, 2, 3])
def test_openmp_build_identical_iterates(orc, k):
    inst = I.small_config(k)
    x1, y1, i1 = orc.solve(inst, tol=1e-6, max_iter=3000)
    try:
        for threads in (2, 5):
            assert orc.use_openmp(True, threads) == threads
            x2, y2, i2 = orc.solve(inst, tol=1e-6, max_iter=3000)
            assert np.array_equal(x1, x2) and np.array_equal(y1, y2), (k, threads)
            assert i1["iters"] == i2["iters"] and i1["inner_total"] == i2["inner_total"]
            assert i1["kkt"] == i2["kkt"]
    finally:
        orc.use_openmp(False)


def test_openmp_build_kkt_and_projection(orc, rng):
    inst = I.small_config(2)
    x, y = rng.normal(size=inst["n"]), rng.normal(size=inst["m"])
    r1 = orc.kkt(inst, x, y)
    p1 = orc.proj_product(inst, x)
    try:
        orc.use_openmp(True, 3)
        assert orc.kkt(inst, x, y) == r1
        assert np.array_equal(orc.proj_product(inst, x), p1)
    finally:
        orc.use_openmp(False)
