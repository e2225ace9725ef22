"""Writes large_qp_2e6_reference.npz: the FP64 oracle's solution of the large sparse QP at 1/100
of the full size (n = 2,000,000, m = 500,000, 10^7 nnz in A, seed 2105), solved to relative
KKT <= 1e-7: the objective and the optimal x at 4,096 fixed indices (Q is positive definite on
this instance, so x* is unique).  Calls only the oracle and the seeded instance generator; the
GPU test compares its own solve of the device-generated copy with these values.

Usage: python tests/golden/make_large_qp_reference.py [threads]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import instances  # noqa: E402
import oracle  # noqa: E402

N, M, SEED = 2_000_000, 500_000, 2105


def sample_indices():
    return np.linspace(0, N - 1, 4096).astype(np.int64)


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    inst = instances.large_qp(n=N, m=M, seed=SEED)
    used = oracle.use_openmp(threads > 0, threads)
    t0 = time.perf_counter()
    x, y, info = oracle.solve(inst, tol=1e-7, max_iter=2_000_000)
    dt = time.perf_counter() - t0
    idx = sample_indices()
    k = info["kkt"]
    np.savez_compressed(os.path.join(HERE, "large_qp_2e6_reference.npz"), idx=idx, x=x[idx],
                        pobj=k["pobj"], dobj=k["dobj"], rel_kkt=k["rel_kkt"], iters=info["iters"],
                        status=info["status"], n=N, m=M, seed=SEED)
    print("status %d iters %d rel_kkt %.3e pobj %.12g (%d threads, %.0f s)"
          % (info["status"], info["iters"], k["rel_kkt"], k["pobj"], used, dt))


if __name__ == "__main__":
    main()
