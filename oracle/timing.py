"""Timing harness for the oracle (test infrastructure: used by bench.py's CPU-baseline and
reference legs).  Runs as a script so the caller can pin the BLAS thread count.

python -m oracle.timing <workload> <n_solves> [max_seconds]
prints one JSON line: setup seconds, per-solve seconds, iterations, threads.
"""
from __future__ import annotations

import json
import os
import sys
import time


def main():
    name = sys.argv[1]
    n = int(sys.argv[2])
    budget = float(sys.argv[3]) if len(sys.argv) > 3 else 1e9
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import workloads as W
    from oracle import dd
    w = W.WORKLOADS[name]()
    t0 = time.perf_counter()
    prob = dd.problem_from_workload(w, thetas=w.thetas[:1])
    s = dd.DDSolver(prob)
    setup = time.perf_counter() - t0
    times, its = [], []
    t_start = time.perf_counter()
    for _ in range(n):
        t = time.perf_counter()
        r = s.solve(tol=1e-10)
        times.append(time.perf_counter() - t)
        its.append(r["iterations"][0])
        if time.perf_counter() - t_start > budget:
            break
    print(json.dumps({"workload": name, "setup_s": setup, "solve_s": times, "iterations": its,
                      "threads": int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1)),
                      "n_dual": s.nd, "n_coarse": s.n2, "l": s.l}))


if __name__ == "__main__":
    main()
