"""Timing harness for the oracle (test infrastructure: used by bench.py's CPU-baseline and
reference legs).  Runs as a script so the caller can pin the BLAS thread count.

python -m oracle.timing <workload>[@cornerN] <n_solves> [max_seconds]
prints one JSON line: setup seconds, per-solve seconds, iterations, threads.
``name@cornerN`` times the N x N corner block of a uniform workload (workloads.corner_block):
a bounded sample with the same element operators, for workloads too large for the oracle.
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
    if "@corner" in name:
        base, n_blk = name.split("@corner")
        w = W.corner_block(W.WORKLOADS[base](), int(n_blk))
    else:
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
    print(json.dumps({"workload": name, "n_elem": w.n_elem, "setup_s": setup, "solve_s": times, "iterations": its,
                      "threads": int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1)),
                      "n_dual": s.nd, "n_coarse": s.n2, "l": s.l}))


if __name__ == "__main__":
    main()
