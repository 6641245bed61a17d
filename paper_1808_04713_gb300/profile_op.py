"""Time the components of one interface-operator application on a named workload.

    python -m paper_1808_04713_gb300.profile_op <workload> [R] [fp64|mixed] [reps] [solves] [opt=value ...]

Factors the workload, runs one solve with R right-hand sides (which sizes the work buffers
and captures the iteration graph), then prints the average milliseconds per application of
pass 1, coarse assembly, coarse solve, pass 2, jump gather and preconditioner, each timed with
CUDA events on the library stream (ddh_profile_op).  With `solves` > 0 it then runs that
many more complete solves (for launch lists of a whole solve).  Arguments of the form
name=value are factor options (ddh_options fields), e.g. edge_launch=1 nd_chains=2 to pin the
launch forms the autotuners pick in a plain run (under a profiler the serialised launches can
make them pick others).  A short fixed command for profilers.
"""
from __future__ import annotations

import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv=None) -> None:
    import torch
    import workloads as W
    from paper_1808_04713_gb300 import ddh

    argv = sys.argv[1:] if argv is None else argv
    opts = {}
    for a in [a for a in argv if "=" in a]:
        k, v = a.split("=", 1)
        opts[k] = float(v) if "." in v or "e" in v else int(v)
    argv = [a for a in argv if "=" not in a]
    name = argv[0] if argv else "plane_16x16"
    w = W.WORKLOADS[name]()
    R = int(argv[1]) if len(argv) > 1 else w.n_rhs
    prec = ddh.PREC_MIXED_FP32 if len(argv) > 2 and argv[2] == "mixed" else ddh.PREC_FP64
    reps = int(argv[3]) if len(argv) > 3 else 3
    solves = int(argv[4]) if len(argv) > 4 else 0
    s = ddh.DDH(0)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(tol=1e-10, precision=prec, **opts)
    b = s.rhs_planewave(w.thetas[:R])
    _, st = s.solve(b, tol=1e-10, allow_noconv=True)
    torch.cuda.synchronize()
    ms = s.profile_op(R, 0 if prec == ddh.PREC_FP64 else 1, reps)
    info = s.info()
    for _ in range(solves):
        _, st = s.solve(b, tol=1e-10, allow_noconv=True)
    torch.cuda.synchronize()
    keys = ["pass1", "coarse_assemble", "coarse_solve", "pass2", "jump_gather", "precond"]
    print(json.dumps({"workload": name, "rhs": R, "precision": "fp64" if prec == ddh.PREC_FP64 else "mixed",
                      "iterations": max(x.iterations for x in st), "coarse_fronts": info.n_coarse_blocks,
                      "ms": {k: round(float(v), 5) for k, v in zip(keys, ms)}}))
    s.close()


if __name__ == "__main__":
    main()
