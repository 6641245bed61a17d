#!/usr/bin/env python
"""Benchmark: Helmholtz DD solves/sec at relative residual 1e-10 (plane_16x16 workload:
16x16 squares, p = 16, k = 100, one plane wave, complex128 -- the plain FP64 GPU method).

One step = one complete solve (RHS resident on the device): the RHS pass g = C^ A^-1 b^,
FGMRES on the dual interface problem to relative residual 1e-10 (every iteration one
preconditioner application and one interface-operator application: local solves, coarse
assembly and solve, jump gather), and the recovery of the element solution.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica of the workload (the path shards by
independent problems: no data-path collective) and rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Helmholtz DD solves/sec at rel. residual 1e-10; mixed+batched vs plain FP64"
COMPARE_WORKLOAD = "random_eps_64"
UNIT = "solves/s"
WORKLOAD = "plane_16x16"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(value: float, device: str) -> float:
    """The largest of `value` over the ranks of the process group (the job's time is its
    slowest replica's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, steps: int, rhs: int, slowest_total_s: float) -> float:
    """Whole-job solves/s of N independent replicas: every rank solves `steps` batches of
    `rhs` right-hand sides; the job takes as long as its slowest rank."""
    return world * steps * rhs / slowest_total_s


def workload_config(R: int, l: int, n_dual: int, n_coarse: int, l2: str, parallelism: str) -> dict:
    """The `config` object of both arms: the timed workload (16 x 16 squares of degree 16,
    k = 100, one plane wave) and the sizes the method derives from it."""
    return {"workload": WORKLOAD, "mesh": "16x16 squares", "p": 16, "k": 100.0, "rhs": R,
            "l": int(l), "n_dual": int(n_dual), "n_coarse": int(n_coarse),
            "dof": int((16 * 16 + 1) ** 2), "precision": "fp64", "l2": l2, "parallelism": parallelism}


def _oracle_timing(name: str, n: int, budget: float, threads: int = 1) -> dict:
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads), CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-m", "oracle.timing", name, str(n), str(budget)],
                         cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (every 10 ms).  Started before the
    warm-up so that it is running when the timed region begins; `mark(t0, t1)` keeps the
    samples taken inside the timed region (wall clock), else the one nearest to it."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.window = None

    def __enter__(self):
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        import datetime
        for line in self.proc.stdout:
            cols = [c.strip() for c in line.split(",")]
            try:
                t = datetime.datetime.strptime(cols[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except (ValueError, IndexError):
                t = time.time()
            self.rows.append((t, cols[1:]))

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        rows = self.rows
        inside = rows
        if self.window and rows:
            t0, t1 = self.window
            inside = [r for r in rows if t0 - 0.01 <= r[0] <= t1 + 0.01]
            if not inside:
                mid = 0.5 * (t0 + t1)
                inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, r in inside:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for n, v in zip(names, r[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_work(info, R: int, p: int, nE: float, nT: float, fp64: bool):
    """Algorithmic FLOPs and HBM bytes per launch of the operator components, Krylov-loop
    form with explicit edge operators: index 0 pass 1 ([S_E^-1; Y^T] r_E), 2 coarse solve
    (dense K^-1), 3 pass 2 (x_E - Y u_T); n_E type-1 edge and n_T type-2 slots per element."""
    E = info.n_elem
    cb = 16 if fp64 else 8
    flops_pass1 = E * R * 8 * (nE * nE + nE * nT)
    bytes_pass1 = E * cb * (nE * nE + nE * nT) + E * R * cb * (2 * nE + nT)
    flops_pass2 = E * R * 8 * nE * nT
    bytes_pass2 = E * cb * nE * nT + E * R * cb * (2 * nE + nT)
    nc = info.n_coarse
    flops_coarse = 8.0 * nc * nc * R
    bytes_coarse = 16.0 * nc * nc + 32.0 * nc * R
    return {0: (flops_pass1, bytes_pass1), 2: (flops_coarse, bytes_coarse), 3: (flops_pass2, bytes_pass2)}


def _mixed_vs_plain(local: int, stream, steps: int) -> dict:
    """Mixed precision (complex64 inner DD, FP64 outer FGMRES on the conforming system) against
    the plain FP64 method on the batched 64x64 workload (p = 20, k = 400, random eps, 8 plane
    waves), both to the same FP64 primal relative residual 1e-10; CUDA events on the library
    stream, right-hand sides resident (the 231 MB of local vectors exceed L2)."""
    import torch
    import workloads as W
    from paper_1808_04713_gb300 import ddh
    w = W.WORKLOADS[COMPARE_WORKLOAD]()
    R = w.n_rhs
    res = {"workload": COMPARE_WORKLOAD, "rhs": R, "tol": 1e-10, "steps": steps}
    for name, prec in (("plain_fp64", ddh.PREC_FP64), ("mixed", ddh.PREC_MIXED_FP32)):
        s = ddh.DDH(local, stream=stream)
        s.set_mesh(w.base_n, w.leaves, w.p)
        s.set_coefficients(w.k, w.eps)
        s.factor(tol=1e-10, precision=prec)
        with torch.cuda.stream(stream):
            b = s.rhs_planewave(w.thetas)
            u = torch.empty_like(b)
        _, st = s.solve(b, tol=1e-10, out=u)
        ts = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            _, st = s.solve(b, tol=1e-10, out=u)
            with torch.cuda.stream(stream):
                e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        pr = s.primal_residual(b, u)
        res[name] = {"value": round(R * len(ts) / sum(ts), 3), "unit": UNIT,
                     "ms_per_solve_batch": round(1e3 * sum(ts) / len(ts), 3),
                     "iterations": max(x.iterations for x in st),
                     "inner_iterations": max(x.inner_iterations for x in st),
                     "max_primal_residual": float(max(pr))}
        s.close()
    res["mixed_over_plain"] = round(res["mixed"]["value"] / res["plain_fp64"]["value"], 3)
    return res


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1808_04713_gb300 import build as B
    B.build()
    import workloads as W
    from paper_1808_04713_gb300 import ddh
    w = W.WORKLOADS[WORKLOAD]()
    stream = torch.cuda.Stream()
    s = ddh.DDH(local, stream=stream)
    s.set_mesh(w.base_n, w.leaves, w.p)
    s.set_coefficients(w.k, w.eps)
    s.factor(tol=1e-10)
    info = s.info()
    R = w.n_rhs
    with torch.cuda.stream(stream):
        b = s.rhs_planewave(w.thetas)
        u = torch.empty_like(b)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    clk = ClockSampler(local).__enter__()        # running before the timed region starts
    for _ in range(args.warmup):
        _, st = s.solve(b, tol=1e-10, out=u)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    times = []
    launches0 = s.kernel_launches()
    iters = []
    t_start = time.time()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()                  # evict L2 (256 MB > 129 MB) between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        _, st = s.solve(b, tol=1e-10, out=u)
        with torch.cuda.stream(stream):
            e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        iters.append(st[0].iterations)
    torch.cuda.synchronize()
    clk.mark(t_start, time.time())
    clk.__exit__(None, None, None)
    launches = s.kernel_launches() - launches0
    total = sum(times)
    if ws > 1:
        total = _max_over_ranks(total, f"cuda:{local}")
    value = aggregate_rate(ws, args.steps, R, total)
    # end-to-end through the public API with pinned host buffers
    bh = torch.empty(b.shape, dtype=b.dtype, pin_memory=True)
    uh = torch.empty(b.shape, dtype=b.dtype, pin_memory=True)
    bh.copy_(b.cpu())
    e2e_t = []
    for _ in range(max(1, args.steps)):
        with torch.cuda.stream(stream):
            flush.zero_()                  # same L2 state as the device-timed steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st_ = s.lib.ddh_solve_host(s.h, bh.data_ptr(), uh.data_ptr(), R, 1e-10, None)
        e2e_t.append(time.perf_counter() - t0)
        assert st_ == 0, s.lib.ddh_last_error(s.h)
    e2e_total = sum(e2e_t)
    if ws > 1:
        e2e_total = _max_over_ranks(e2e_total, f"cuda:{local}")
    e2e_value = aggregate_rate(ws, len(e2e_t), R, e2e_total)
    # correctness of the timed result
    pr = s.primal_residual(b, u)
    # live per-component timing of the operator (CUDA events on the library stream)
    comp = s.profile_op(R, ddh.PREC_FP64, reps=20)
    m = s.lib
    nE = (4 * (w.p[0] - info.l))
    nT = 4 + 4 * (info.l - 1)
    work = algorithmic_work(info, R, int(w.p[0]), nE, nT, True)
    names = {0: "pass1 (edge operators: [S_E^-1; Y^T] r_E)", 2: "coarse solve (dense K^-1 GEMV, FP64)",
             3: "pass2 (edge operators: x_E - Y u_T)"}
    dom = max(work, key=lambda i: comp[i])
    fl, by = work[dom]
    fp64_peak = 1250.0         # GFLOP/s... expressed in TFLOP/s below
    achieved_tf = fl / (comp[dom] * 1e-3) / 1e12
    # dram__bytes_read + dram__bytes_write of one dense-K^-1 GEMV launch (plane_16x16; k_gemv, and
    # k_gemv1 reads the same 59.09 MB) from the ncu captures summarised in
    # profiles/launches_plane16x16_fp64.md; unknown for other kernels
    traffic = 59092224 + 2816 if (dom == 2 and WORKLOAD == "plane_16x16" and R == 1) else None
    roof = {"kernel": names[dom], "bound": "alu", "achieved": round(achieved_tf, 4),
            "peak": 1.25, "unit": "TFLOP/s", "frac": round(achieved_tf / 1.25, 4), "traffic": traffic,
            "algorithmic_bytes": int(by),
            "peak_source": "fallback: nominal GB300 FP64 1.25 TFLOP/s (measured DGEMM 1.10)",
            "achieved_hbm_GBs": round(by / (comp[dom] * 1e-3) / 1e9, 1),
            "component_ms": {"pass1": comp[0], "coarse_assemble": comp[1], "coarse_solve": comp[2],
                             "pass2": comp[3], "jump_gather": comp[4], "precond": comp[5]}}
    clocks = clk.summary()
    compare = None
    if not args.no_compare:
        compare = _mixed_vs_plain(local, stream, 2)
    out = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            o = _oracle_timing(WORKLOAD, 6, 20.0, threads=1)
            per = statistics.mean(o["solve_s"])
            cpu = {"value": round(1.0 / per, 4), "unit": UNIT, "cores": o["threads"], "kind": "oracle",
                   "sample": f"oracle DD solve of {WORKLOAD} (1 RHS, tol 1e-10) repeated {len(o['solve_s'])}x "
                             f"after a {o['setup_s']:.1f}s setup, single BLAS thread; "
                             f"{o['iterations'][0]} FGMRES iterations"}
        out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 4),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
               "data": "synthetic plane-wave impedance data (closed form)",
               "config": workload_config(R, info.l, info.n_dual, info.n_coarse,
                                         "flushed (256 MB write) between timed steps", f"replicas x{ws}"),
               "iterations": iters[-1] if iters else None, "primal_residual": float(pr[0]),
               "dof_per_s": round(value * (16 * 16 + 1) ** 2, 1),
               "e2e": {"value": round(e2e_value, 3), "unit": UNIT,
                       "h2d_bytes_per_step": int(16 * R * info.n_local),
                       "d2h_bytes_per_step": int(16 * R * info.n_local)},
               "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
               "mixed_vs_plain": compare}
        print(json.dumps(out))
    s.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    n = max(1, args.steps + args.warmup)
    o = _oracle_timing(WORKLOAD, n, 150.0, threads=1)
    ts = o["solve_s"][min(args.warmup, len(o["solve_s"]) - 1):]
    per = statistics.mean(ts)
    val = 1.0 / per
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 5), "unit": UNIT, "n_gpus": ws,
           "steps": len(ts), "warmup": args.warmup, "ms_per_step": round(1e3 * per, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic plane-wave impedance data (closed form)",
           "config": workload_config(1, o["l"], o["n_dual"], o["n_coarse"], "host CPU run (no device L2)",
                                     "oracle on rank 0"),
           "cpu_baseline": {"value": round(val, 5), "unit": UNIT, "cores": o["threads"], "kind": "oracle",
                            "sample": f"oracle DD solve of {WORKLOAD}, {len(ts)} timed solves, single BLAS thread"},
           "e2e": {"value": round(val, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the mixed-vs-plain comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
