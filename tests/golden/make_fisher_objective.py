"""Writes fisher_10000x1000_objective.txt: the FP64 oracle's optimal objective of the full
Fisher-market workload (10,000 buyers x 1,000 goods, density 0.05, seed 1003, slice
blocks), solved to relative KKT <= 1e-7.  Calls only the oracle and the seeded instance
generator; the GPU test compares its own solve's objective with this value.

Usage: python tests/golden/make_fisher_objective.py [threads]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import instances  # noqa: E402
import oracle  # noqa: E402


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    inst = instances.fisher_market(n_buyers=10_000, n_goods=1000, density=0.05, seed=1003)
    used = oracle.use_openmp(threads > 0, threads)
    t0 = time.perf_counter()
    _, _, info = oracle.solve(inst, tol=1e-7, max_iter=2_000_000)
    dt = time.perf_counter() - t0
    k = info["kkt"]
    with open(os.path.join(HERE, "fisher_10000x1000_objective.txt"), "w") as f:
        f.write("# FP64 oracle solve of instances.fisher_market(10000, 1000, 0.05, seed 1003), tol 1e-7\n")
        f.write("# written by tests/golden/make_fisher_objective.py (%d threads, %.0f s)\n" % (used, dt))
        f.write("status %d\niters %d\nrel_kkt %.6e\npobj %.17g\ndobj %.17g\n"
                % (info["status"], info["iters"], k["rel_kkt"], k["pobj"], k["dobj"]))
    print(open(os.path.join(HERE, "fisher_10000x1000_objective.txt")).read())


if __name__ == "__main__":
    main()
