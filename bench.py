#!/usr/bin/env python3
"""Time to 1e-4 relative KKT on one GB300 (and the FP64 plain-PDHG comparison).

Workload (default): the SOCP/QCQP mix -- n = 200,000 coordinates (100,000
nonnegative, 2,000 second-order cones of dimension U[10,50], 500 rotated
second-order cones of dimension U[3,20], the rest free), m = 100,000 equality
rows with about 10 N(0,1) entries per column, Q = diag(lognormal(0,1)) + R'R
with R 20 x n, feasible b.  Seeded synthetic data (Philox, seed 1002).

A step is one complete solve through the C ABI: cqp_setup (rescaling,
transpose, norm estimate) from device-resident FP64 inputs, then cqp_solve to
relative KKT <= 1e-4 (FP32 iterates, FP64 reductions and cone roots), outputs
left on the device.  `value` is the mean time per solve (seconds, lower is
better).  L2 is flushed (256 MB write) before every step, outside the timed
event pair.  `e2e` repeats the solve from pinned host buffers with the
host->device copies of the inputs and the device->host copy of (x, y) inside
the timed region.  The FP64 plain-PDHG run (same code, precision = all FP64,
cold start) is timed once as the comparison the metric names.

The line also carries:
  roofline      algorithmic bytes per solve (the per-unit figures of the scope table: the two
                sparse products per outer iteration, R, R' or P and eight n-vectors per inner
                step) over the solver kernel's CUDA-event time, against the measured HBM peak,
                with `traffic` (ncu DRAM bytes per solve from profiles/, when captured on the
                current kernel sources) and `l2` (the same rate against a measured copy between
                two L2-resident 32 MB buffers: this workload's working set stays in L2);
  large         the HBM-bound workload: the large sparse QP (n = 2e8, m = 5e7, 1e9 nnz,
                generated in device memory), one setup + solve to 1e-4 with its own roofline;
  cpu_baseline  the FP64 oracle solving the same instance to 1e-4 on the host: the OpenMP
                build on every core (value) and the single-threaded build (single_thread).

With --gpus N under torchrun each rank solves its own instance (seed + rank):
replicas, no collectives; rank 0 prints the max-over-ranks time.
--impl reference times the FP64 CPU oracle (OpenMP build, every host core, one full solve
to 1e-4 per step) instead.

Other workloads (not the default line):
  --workload portfolio  4,096 uneven portfolio QPs solved in one batched launch
                        (setup + solve of the whole batch per step); with
                        --ws-train N a warm-start network is first trained on N
                        solved instances and the warm-started step is timed too.
  --workload large      the large sparse QP (n = --large-n, m = n/4, 20 nnz per
                        row), generated in device memory; setup + solve per step;
                        --matrix-bf16 2 stores A, A' and P as BF16 (the rounded problem).
  --workload gemm       the warm-start network's BF16 GEMMs at the training shape.
  --workload spmv       the sparse product in each layout (CSR row widths, merge path, sliced
                        ELL) on the large QP's A and an A'-shaped matrix at a tenth of its size
                        (--large-n 2e9: full size).
  --workload lasso      a Lasso with the shape and density of rcv1_test (677,399 x 47,236,
                        density 1.55e-3), reformulated by frontends.lasso_to_qp; setup + solve.
  --workload qcqp       a synthetic convex QCQP (n = 200,000, 50,000 linear rows, 50 quadratic
                        constraints of rank 50), reformulated by frontends.qcqp_to_qsocp.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-4 rel KKT vs FP64 plain PDHG on 1 GB300; SpMV+prox HBM GB/s"
WORKLOAD = ("socp_mix: n=200000 (100000 nonneg, 2000 SOC dim U[10,50], 500 RSOC dim U[3,20], free rest), "
            "m=100000, ~10 nnz/col N(0,1), Q=diag(lognormal)+R'R rank 20, seed 1002")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _l2_copy_gbs(torch, mb=32, reps=50):
    """Bandwidth of a copy whose source and destination (2 x 32 MB) stay in the 129 MB L2: the
    ceiling for a loop whose working set is L2-resident (bytes read + written per copy)."""
    n = mb * 1024 * 1024 // 4
    a = torch.ones(n, device="cuda")
    b = torch.empty_like(a)
    for _ in range(10):
        b.copy_(a)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.copy_(a)
        a.copy_(b)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / (2 * reps)
    return 2.0 * n * 4 / ms / 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(n, m, nnz, iters, inner_total, k=0, pnnz=0, esize=4, isize=4, check_every=64, vsize=None):
    """Bytes the method must move per solve, with the per-unit figures of the scope table's
    measurement section (each array element counted once per pass):
      per outer iteration, the two sparse products A'y (n rows) and A x (m rows):
          values + indices (nnz (esize + isize)) + row pointers + gathered operand + output;
      per inner BB step: R and R' (2 k n esize), the rows of a sparse P (pnnz (esize + isize) plus
          row pointers) and eight n-vectors;
      per KKT check (every check_every iterations): the same two sparse products again.
    vsize: bytes of a stored matrix value of A, A' and P (default esize; 2 with BF16 storage)."""
    vs = esize if vsize is None else vsize
    spmv_at = nnz * (vs + isize) + (n + 1) * isize + m * esize + n * esize
    spmv_a = nnz * (vs + isize) + (m + 1) * isize + n * esize + m * esize
    per_iter = spmv_at + spmv_a
    per_inner = 2 * k * n * esize + (pnnz * (vs + isize) + (n + 1) * isize if pnnz else 0) + 8 * n * esize
    checks = iters // check_every + 1
    return iters * per_iter + inner_total * per_inner + checks * per_iter


def inst_bytes(inst, res, esize=4):
    nnz = int(inst["a_rowptr"][-1])
    k = 0 if inst.get("q_R") is None else int(inst["q_R"].shape[0])
    pnnz = 0 if inst.get("p_rowptr") is None else int(inst["p_rowptr"][-1])
    return algorithmic_bytes(inst["n"], inst["m"], nnz, res["iters"], res["inner_total"], k, pnnz, esize)


SOLVER_SOURCES = ("common.cuh", "cones.cuh", "solver.cuh", "solver_impl.cuh", "kernels.inc", "solver_grid_f32.cu")


def _source_hash():
    """Hash of the sources that make up pdhg_grid_kernel<float>."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2608_09159_gb300", "csrc")
    for f in SOLVER_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(workload="socp_mix"):
    """DRAM bytes per solve of the solver kernel from the committed ncu record of the workload,
    if it was captured on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "pdhg_kernel_%s.json" % workload)
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != _source_hash():
        return None
    return d.get("dram_bytes_per_solve")


def _device_inst(inst, torch):
    out = {}
    for k, v in inst.items():
        if hasattr(v, "dtype") and hasattr(v, "shape") and k in (
                "a_rowptr", "a_colind", "a_val", "c", "b", "q_diag", "q_R", "q_D", "p_rowptr", "p_colind", "p_val",
                "blk_type", "blk_start", "blk_dim", "blk_alpha", "row_lo", "row_hi", "x_lo", "x_hi"):
            import numpy as np
            dt = {"a_colind": np.int32, "p_colind": np.int32, "blk_type": np.int32}.get(k, v.dtype)
            out[k] = torch.from_numpy(np.ascontiguousarray(v, dtype=dt)).cuda()
        else:
            out[k] = v
    return out


def _pinned_inst(inst, torch):
    import numpy as np
    out = dict(inst)
    for k in ("a_rowptr", "a_colind", "a_val", "c", "b", "q_diag", "q_R", "q_D", "blk_type", "blk_start", "blk_dim",
              "blk_alpha"):
        v = inst.get(k)
        if v is None:
            continue
        dt = {"a_colind": np.int32, "blk_type": np.int32}.get(k, v.dtype)
        t = torch.from_numpy(np.ascontiguousarray(v, dtype=dt)).pin_memory()
        out[k] = t.numpy()
        out["_pin_" + k] = t
    return out


def max_over_ranks(value, world):
    """The largest of the ranks' values (the job's time is its slowest replica's).  Uses the
    process group's backend: a CUDA tensor under NCCL, a host tensor under gloo."""
    if world <= 1:
        return value
    import torch
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def make_instance(args, rank):
    import instances
    if args.small:
        return instances.socp_mix(n=20000, n_nonneg=10000, n_soc=200, n_rsoc=50, m=10000, seed=1002 + 1000 * rank)
    return instances.socp_mix(seed=1002 + 1000 * rank)


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2608_09159_gb300 as g
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    g.build()
    g.lib()
    inst = make_instance(args, rank)
    dinst = _device_inst(inst, torch)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    opts = dict(precision=0, tol=1e-4, max_iter=200000, time_limit_s=600.0)

    def one_solve(src, device, out_device, **kw):
        s = g.Solver(src, device=device, **{**opts, **kw})
        x, y, res = s.solve(out_device=out_device)
        s.close()
        return x, y, res

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        flush.fill_(1.0)
        one_solve(dinst, False, True)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    times, results = [], []
    launches0 = g.cqp_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, y, res = one_solve(dinst, False, True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        results.append(res)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    launches = g.cqp_kernel_launches() - launches0
    clk = clocks.stop()
    step_s = statistics.mean(times)
    step_s = max_over_ranks(step_s, world)
    res = results[-1]
    # parity of the timed solution, measured independently on the host (rank 0, FP64 oracle)
    kkt_check = None
    if rank == 0 and not args.no_oracle:
        import oracle
        kkt_check = oracle.kkt(inst, x.double().cpu().numpy(), y.double().cpu().numpy())["rel_kkt"]

    # e2e: the same solve from pinned host buffers, copies inside the timed region
    pinst = _pinned_inst(inst, torch)
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xe, ye, rese = one_solve(pinst, False, False)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    n, m = inst["n"], inst["m"]
    nnz = int(inst["a_rowptr"][-1])
    k = int(inst["q_R"].shape[0])
    h2d = (m + 1) * 8 + nnz * (4 + 8) + 2 * n * 8 + m * 8 + k * n * 8 + k * k * 8 + \
        len(inst["blk_type"]) * (4 + 8 + 8 + 8)
    d2h = (n + m) * 8

    # FP64 plain PDHG (same code, all FP64, cold start)
    fp64 = None
    if args.fp64_steps > 0:
        ft = []
        for _ in range(args.fp64_steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, r64 = one_solve(dinst, False, True, precision=1)
            e1.record(stream)
            e1.synchronize()
            ft.append(e0.elapsed_time(e1) / 1e3)
        fp64 = {"time_s": statistics.mean(ft), "iters": r64["iters"], "inner": r64["inner_total"],
                "rel_kkt": r64["kkt"]["rel_kkt"], "rc": r64["rc"]}

    peaks, src = _peaks()
    alg = inst_bytes(inst, res)
    kern_s = res["kernel_ms"] / 1e3
    achieved = alg / kern_s / 1e9 if kern_s > 0 else None
    traffic = _ncu_traffic()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": (achieved / peaks["hbm_gbs"]) if achieved else None, "traffic": traffic,
            "peak_source": src, "kernel": "pdhg_grid_kernel<float, false>", "algorithmic_bytes_per_solve": alg,
            "kernel_s_per_solve": kern_s}
    # the working set of this workload (about 60 MB) stays in L2: the same achieved rate against a
    # measured L2-resident copy, beside the HBM fraction
    l2 = _l2_copy_gbs(torch)
    roof["l2"] = {"peak": l2, "unit": "GB/s", "frac": (achieved / l2) if achieved else None,
                  "method": "copy between two 32 MB device buffers (L2-resident), bytes read + written, CUDA events"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(inst, args)
    # the HBM half of the metric: the large sparse QP (one setup + solve, no warm-up) on rank 0
    large = None
    if rank == 0 and world == 1 and not args.no_large and not args.small:
        del dinst
        torch.cuda.empty_cache()
        large = large_solve(args, 1, 0, flush)

    line = {
        "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "precision": "FP32 iterates, matrices and SOC roots; FP64 reductions, KKT, restart control and RSOC/exp/pow roots", "data": "synthetic (Philox-seeded)",
        "config": {"workload": WORKLOAD, "n": n, "m": m, "nnz": nnz, "tol": 1e-4, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed before every step (256 MB write)", "inputs": "device-resident FP64 (HBM)"},
        "e2e": {"value": statistics.mean(e2e_times), "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "large": large,
        "cpu_baseline": cpu,
        "fp64_plain_pdhg": fp64,
        "speedup_vs_fp64": (fp64["time_s"] / step_s) if fp64 else None,
        "solve": {"iters": res["iters"], "restarts": res["restarts"], "inner_total": res["inner_total"],
                  "rel_kkt": res["kkt"]["rel_kkt"], "oracle_rel_kkt": kkt_check, "setup_ms": res["setup_ms"],
                  "solve_ms": res["solve_ms"], "kernel_ms": res["kernel_ms"], "iters_per_s": res["iters"] / step_s,
                  "step_times_s": times, "wall_s": wall},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def _timed(fn, steps, warmup, flush, counter=None):
    """W untimed warm-up steps, then `steps` steps each bracketed by CUDA events on the current
    stream with an L2 flush before it.  Returns (step times, last output, library kernel launches
    inside the timed steps as read from `counter`, or None)."""
    import torch
    for _ in range(warmup):
        flush.fill_(1.0)
        fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times, out = [], None
    c0 = counter() if counter else 0
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times, out, (counter() - c0 if counter else None)


def run_portfolio(args):
    import numpy as np
    import torch

    import instances
    import paper_2608_09159_gb300 as g
    from paper_2608_09159_gb300 import warmstart as W
    g.build()
    g.lib()
    batch = instances.portfolio_batch()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    opts = dict(precision=0, tol=1e-4, max_iter=100000, time_limit_s=600.0)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    times, (x, y, per, res), launches = _timed(lambda: W.solve_batch(batch, None, **opts), args.steps, args.warmup,
                                               flush, g.cqp_kernel_launches)
    its = np.array([r["iters"] for r in per])
    line = {"metric": "time to 1e-4 rel KKT on every instance of the batch", "value": statistics.mean(times),
            "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (Philox-seeded)",
            "config": {"workload": "portfolio_batch: 4096 instances, n_i ~ U[50,2000] assets, k_i ~ U[10,50] "
                                   "factors, seed 1004", "n": batch["n"], "m": batch["m"],
                       "nnz": int(batch["a_rowptr"][-1]), "l2": "flushed before every step (256 MB write)",
                       "inputs": "host arrays copied to the device inside the step"},
            "batch": {"converged": int(sum(r["rc"] == 0 for r in per)), "count": len(per),
                      "iters_mean": float(its.mean()), "iters_max": int(its.max()),
                      "inner_total": res["inner_total"], "kernel_ms": res["kernel_ms"], "setup_ms": res["setup_ms"],
                      "max_rel_kkt": max(r["kkt"]["rel_kkt"] for r in per)},
            "gpu_launches": launches}
    if args.ws_train > 0:
        data = W.TrainingSet()
        per_batch = min(4096, args.ws_train)
        nb = (args.ws_train + per_batch - 1) // per_batch
        for k in range(nb):
            tb = instances.portfolio_batch(count=per_batch, seed=11001 + k)
            xt, yt, pt, rt = W.solve_batch(tb, None, **opts)
            data.add(tb, xt.cpu().numpy(), yt.cpu().numpy())
        net = W.WarmStartNet(seed=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W.train(net, data, steps=args.ws_steps, instances=256, lr=1e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del data
        wt, (xw, yw, pw, rw), _ = _timed(lambda: W.solve_batch(batch, net, **opts), args.steps, args.warmup, flush)
        iw = np.array([r["iters"] for r in pw])
        line["warm_start"] = {"value": statistics.mean(wt), "unit": "s", "trained_on": nb * per_batch,
                              "train_steps": args.ws_steps, "train_s": t_train, "iters_mean": float(iw.mean()),
                              "kernel_ms": rw["kernel_ms"], "converged": int(sum(r["rc"] == 0 for r in pw)),
                              "max_rel_kkt": max(r["kkt"]["rel_kkt"] for r in pw)}
    line["clocks"] = clocks.stop()
    print(json.dumps(line), flush=True)


LARGE_DESC = ("large_qp: n=%d nonneg, m=%d, 20 nnz per row (about 5 per column) N(0,1), Q = diag(U[0,1]) + "
              "Laplacian of a perfect matching (|N(0,1)| weights), c ~ N(0,1), b = A|N(0,1)|, seed 1005")


def large_solve(args, steps, warmup, flush):
    """The large sparse QP generated in device memory; each step is cqp_setup + cqp_solve to
    relative KKT <= 1e-4 from the device-resident FP64 inputs (FP32 iterates)."""
    import torch

    import paper_2608_09159_gb300 as g
    from instances import gpu as G
    n = int(args.large_n)
    n -= n % 2
    m = n // 4
    inst = G.large_qp_device(n=n, m=m, seed=1005)
    torch.cuda.synchronize()

    bf = int(getattr(args, "matrix_bf16", 0))

    def step():
        s = g.Solver(inst, device=True, precision=0, tol=1e-4, max_iter=1000000, time_limit_s=900.0, matrix_bf16=bf)
        out = s.solve(out_device=True)
        s.close()
        return out

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    times, (x, y, res), launches = _timed(step, steps, warmup, flush, g.cqp_kernel_launches)
    clk = clocks.stop()
    nnz, pnnz = m * 20, 2 * n
    # mode 2 (A and P in BF16) is the one this workload takes: its rounded P stays a diagonal plus
    # a weighted matching Laplacian, positive semidefinite
    alg = algorithmic_bytes(n, m, nnz, res["iters"], res["inner_total"], 0, pnnz, vsize=2 if bf else None)
    peaks, src = _peaks()
    kern_s = res["kernel_ms"] / 1e3
    achieved = alg / kern_s / 1e9
    del inst, x, y
    torch.cuda.empty_cache()
    return {"value": statistics.mean(times), "unit": "s", "steps": steps, "warmup": warmup,
            "workload": LARGE_DESC % (n, m), "n": n, "m": m, "nnz": nnz, "pnnz": pnnz,
            "inputs": "device-resident FP64, generated in device memory (Philox, index-addressed)",
            "matrix_values": ("BF16 (A and P rounded to BF16 at setup; the rounded problem is solved and "
                              "measured)") if bf else "FP32",
            "gpu_launches": launches,
            "solve": {"rc": res["rc"], "iters": res["iters"], "inner_total": res["inner_total"],
                      "restarts": res["restarts"], "rel_kkt": res["kkt"]["rel_kkt"], "setup_ms": res["setup_ms"],
                      "kernel_ms": res["kernel_ms"], "step_times_s": times},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None if bf else _ncu_traffic("large"),
                         "peak_source": src, "kernel": "pdhg_grid_kernel<float, false>",
                         "algorithmic_bytes_per_solve": alg, "kernel_s_per_solve": kern_s},
            "clocks": clk}


def run_large(args):
    import torch

    import paper_2608_09159_gb300 as g
    g.build()
    g.lib()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rec = large_solve(args, args.steps, args.warmup, flush)
    line = {"metric": "time to 1e-4 rel KKT", "value": rec["value"], "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["value"] * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (Philox-seeded, generated in device memory)",
            "config": {"workload": rec["workload"], "n": rec["n"], "m": rec["m"], "nnz": rec["nnz"],
                       "pnnz": rec["pnnz"], "inputs": rec["inputs"], "matrix_values": rec["matrix_values"]},
            "gpu_launches": rec["gpu_launches"], "solve": rec["solve"], "roofline": rec["roofline"],
            "clocks": rec["clocks"]}
    print(json.dumps(line), flush=True)


def run_frontend(args):
    """Time to 1e-4 on a front-end workload: one step = cqp_setup_general + cqp_solve from
    device-resident FP64 inputs (the reformulation itself is host-side model building and runs
    once, outside the timed region)."""
    import numpy as np
    import torch

    import instances
    import paper_2608_09159_gb300 as g
    from paper_2608_09159_gb300 import frontends as F
    g.build()
    g.lib()
    t0 = time.perf_counter()
    if args.workload == "lasso":
        L = instances.lasso_problem()
        inst, _ = F.lasso_to_qp((L["a_rowptr"], L["a_colind"], L["a_val"]), L["b"], L["lam"], m=L["m"], n=L["n"])
        desc = ("lasso (rcv1_test shape, synthetic values): A %d x %d, %d nnz, lam = 0.01 ||A'b||_inf, seed 1006; "
                "QP reformulation n=%d, m=%d" % (L["m"], L["n"], int(L["a_rowptr"][-1]), inst["n"], inst["m"]))
    else:
        Q = instances.qcqp_problem(n=200_000, m_lin=50_000, p=50, k=50, k0=20, c_nnz=2000)
        inst, _ = F.qcqp_to_qsocp(Q["n"], Q["c0"], Q["quad"], q0_diag=Q["q0_diag"], q0_R=Q["q0_R"], A=Q["A"],
                                  row_lo=Q["row_lo"], row_hi=Q["row_hi"], x_lo=Q["x_lo"], x_hi=Q["x_hi"])
        desc = ("qcqp: n=200000 box-bounded, 50000 linear rows (10 nnz), 50 quadratic constraints of rank 50 "
                "(20 nnz per factor row), Q0 = diag + R0'R0 rank 20, seed 1007; QSOCP n=%d, m=%d"
                % (inst["n"], inst["m"]))
    t_build = time.perf_counter() - t0
    dinst = _device_inst(inst, torch)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():
        s = g.Solver(dinst, precision=0, tol=1e-4, max_iter=1000000, time_limit_s=900.0)
        out = s.solve(out_device=True)
        s.close()
        return out

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    times, (x, y, res), launches = _timed(step, args.steps, args.warmup, flush, g.cqp_kernel_launches)
    alg = inst_bytes(inst, res)
    peaks, src = _peaks()
    achieved = alg / (res["kernel_ms"] / 1e3) / 1e9
    kkt_check = None
    if not args.no_oracle:
        import oracle
        kkt_check = oracle.kkt(inst, x.double().cpu().numpy(), y.double().cpu().numpy())["rel_kkt"]
    line = {"metric": "time to 1e-4 rel KKT", "value": statistics.mean(times), "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (Philox-seeded)",
            "config": {"workload": desc, "n": inst["n"], "m": inst["m"], "nnz": int(inst["a_rowptr"][-1]),
                       "inputs": "device-resident FP64", "l2": "flushed before every step (256 MB write)",
                       "model_build_s": t_build},
            "gpu_launches": launches,
            "solve": {"rc": res["rc"], "iters": res["iters"], "inner_total": res["inner_total"],
                      "restarts": res["restarts"], "rel_kkt": res["kkt"]["rel_kkt"], "oracle_rel_kkt": kkt_check,
                      "setup_ms": res["setup_ms"], "kernel_ms": res["kernel_ms"], "step_times_s": times},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                         "kernel": "pdhg_grid_kernel<float, true>", "algorithmic_bytes_per_solve": alg},
            "clocks": clocks.stop()}
    print(json.dumps(line), flush=True)


def run_gemm(args):
    """The warm-start network's GEMMs at the training shape (262,144 asset rows, width 512)."""
    import torch

    import paper_2608_09159_gb300 as g
    g.build()
    g.lib()
    rows, H = 262144, 512
    gen = torch.Generator(device="cuda").manual_seed(0)
    H1 = torch.randn(rows, H, device="cuda", generator=gen).to(torch.bfloat16)
    Wt = torch.randn(H, H, device="cuda", generator=gen).to(torch.bfloat16)
    out = torch.empty(rows, H, dtype=torch.bfloat16, device="cuda")
    gw = torch.zeros(H, H, dtype=torch.float32, device="cuda")
    bias = torch.zeros(H, device="cuda")
    # (name, call, kernel): the forward and dH1 products are A B' forms (tcgen05, tensor memory);
    # the weight gradient is A' B with split K (warp-level mma kernel)
    cases = [
        ("forward Z2 = H1 (W2')' (+bias, ReLU, BF16 out)",
         lambda: g.cqp_gemm_bf16(0, 1, rows, H, H, H1.data_ptr(), H, Wt.data_ptr(), H, out.data_ptr(), H,
                                 bias.data_ptr(), 2), "k_gemm_tc_persistent"),
        ("backward dH1 = dZ2 W2' (BF16 out)",
         lambda: g.cqp_gemm_bf16(0, 1, rows, H, H, H1.data_ptr(), H, Wt.data_ptr(), H, out.data_ptr(), H, None, 4),
         "k_gemm_tc_persistent"),
        ("forward Z2 = H1 W2, untransposed weight (+bias, ReLU, BF16 out)",
         lambda: g.cqp_gemm_bf16(0, 0, rows, H, H, H1.data_ptr(), H, Wt.data_ptr(), H, out.data_ptr(), H,
                                 bias.data_ptr(), 2), "k_gemm_bf16"),
        ("backward dW2 += H1' dZ2 (split-K, FP32 atomics)",
         lambda: g.cqp_gemm_bf16(1, 0, H, H, rows, H1.data_ptr(), H, out.data_ptr(), H, gw.data_ptr(), H, None, 3,
                                 128), "k_gemm_bf16")]
    peaks, src = _peaks()
    res = {}
    launches = 0
    tc0 = g.lib().cqp_gemm_tc_launches()
    for name, fn, kern in cases:
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        c0 = g.cqp_kernel_launches()
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        launches += g.cqp_kernel_launches() - c0
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms": ms, "tflops": 2.0 * rows * H * H / ms / 1e9, "kernel": kern}
    g.cqp_gemm_check()
    tc_launches = g.lib().cqp_gemm_tc_launches() - tc0
    best_name = max(res, key=lambda k: res[k]["tflops"])
    best = res[best_name]["tflops"]
    line = {"metric": "warm-start GEMM throughput", "value": statistics.mean(v["tflops"] for v in res.values()),
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "bf16 (FP32 accumulation)", "data": "synthetic",
            "config": {"workload": "MLP layer 2: 262144 x 512 x 512",
                       "l2": "operands larger than L2 (268 MB of BF16 activations per GEMM)"},
            "gemms": res, "gpu_launches": launches, "tensor_memory_gemm_launches": tc_launches,
            "roofline": {"bound": "tensor", "achieved": best, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": best / peaks["bf16_tflops"], "peak_source": src, "kernel": res[best_name]["kernel"],
                         "case": best_name}}
    print(json.dumps(line), flush=True)


def run_spmv(args):
    """The sparse product y = A x in each layout of the library, on the large QP's A (20 entries per
    row) and on a matrix with A''s shape and row-length profile (n rows, Poisson(5) entries per row,
    random columns over m), at n = --large-n / 10 by default (2e7: 1e8 entries, operands well
    above L2).  Throughput in algorithmic bytes: entries (value + index), row pointers, the output
    and one pass over the input vector."""
    import torch

    import paper_2608_09159_gb300 as g
    from instances import gpu as G
    g.build()
    g.lib()
    n = int(args.large_n / 10)
    n -= n % 2
    m = n // 4
    inst = G.large_qp_device(n=n, m=m, seed=1005)
    A = (m, n, inst["a_rowptr"].to(torch.int32), inst["a_colind"], inst["a_val"].to(torch.float32))
    del inst
    gen = torch.Generator(device="cuda").manual_seed(11)
    lens = torch.poisson(torch.full((n,), 5.0, device="cuda"), generator=gen).to(torch.int64)
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    rp[1:] = torch.cumsum(lens, 0)
    nz = int(rp[-1])
    T = (n, m, rp.to(torch.int32), torch.randint(0, m, (nz,), device="cuda", generator=gen, dtype=torch.int32),
         torch.randn(nz, device="cuda", generator=gen))
    del lens, rp
    peaks, src = _peaks()
    res = {}
    launches = 0
    for mname, (rows, cols, rpt, cit, vt) in (("A (m x n, 20 per row)", A), ("A'-shaped (n x m, Poisson(5) per row)", T)):
        x = torch.randn(cols, device="cuda", generator=gen)
        y = torch.empty(rows, device="cuda")
        nnz = int(vt.numel())
        alg = nnz * 8 + (rows + 1) * 4 + rows * 4 + cols * 4
        sell = g.Sell(0, rows, cols, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr())
        variants = {"csr 1 lane/row": lambda: g.cqp_spmv(0, rows, cols, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(),
                                                        x.data_ptr(), y.data_ptr(), 1),
                    "csr 1 lane/row, 4 rows in flight": lambda: g.cqp_spmv(0, rows, cols, rpt.data_ptr(), cit.data_ptr(),
                                                                          vt.data_ptr(), x.data_ptr(), y.data_ptr(), -1),
                    "csr 4 lanes/row": lambda: g.cqp_spmv(0, rows, cols, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(),
                                                         x.data_ptr(), y.data_ptr(), 4),
                    "csr 32 lanes/row": lambda: g.cqp_spmv(0, rows, cols, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(),
                                                          x.data_ptr(), y.data_ptr(), 32),
                    "merge path": lambda: g.cqp_spmv_merge(0, rows, cols, rpt.data_ptr(), cit.data_ptr(), vt.data_ptr(),
                                                           x.data_ptr(), y.data_ptr()),
                    "sliced ELL-32": lambda: sell.spmv(x.data_ptr(), y.data_ptr())}
        out = {}
        for vname, fn in variants.items():
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            c0 = g.cqp_kernel_launches()
            ts = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            launches += g.cqp_kernel_launches() - c0
            ms = statistics.median(ts)
            out[vname] = {"ms": ms, "gbs": alg / ms / 1e6}
        out["sell_stored_over_nnz"] = sell.stored / nnz
        sell.close()
        res[mname] = {"rows": rows, "cols": cols, "nnz": nnz, "algorithmic_bytes": alg, "variants": out}
    best = max((v["gbs"], mn, vn) for mn, r in res.items() for vn, v in r["variants"].items() if isinstance(v, dict))
    line = {"metric": "SpMV throughput (algorithmic bytes)", "value": best[0], "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (Philox / torch generator, device memory)",
            "config": {"workload": "large QP A and an A'-shaped matrix at n = %d, m = %d" % (n, m),
                       "l2": "operands larger than L2 (no flush needed)"},
            "matrices": res, "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": best[0], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": best[0] / peaks["hbm_gbs"], "peak_source": src, "case": "%s, %s" % (best[1], best[2])}}
    print(json.dumps(line), flush=True)


def _oracle_solve_timed(inst, threads):
    """One FP64 oracle solve of the instance to relative KKT <= 1e-4 (threads = 0: the
    single-threaded build, else the OpenMP build with that many threads)."""
    import oracle
    used = oracle.use_openmp(threads > 0, threads)
    try:
        t0 = time.perf_counter()
        _, _, info = oracle.solve(inst, tol=1e-4, max_iter=200000)
        dt = time.perf_counter() - t0
    finally:
        oracle.use_openmp(False)
    return dt, used, info


def cpu_baseline(inst, args):
    """The FP64 oracle, as it stands, solving the same instance to relative KKT <= 1e-4 on the
    host cores: once with the single-threaded build and once with the OpenMP build of the same
    source on every core (the two builds return identical iterates)."""
    import oracle
    oracle.build()
    oracle.build(omp=True)
    nproc = os.cpu_count() or 1
    t_all, used, info = _oracle_solve_timed(inst, nproc)
    out = {"value": t_all, "unit": "s", "cores": used, "kind": "oracle", "nproc": nproc,
           "sample": "one full solve of the same instance to rel-KKT <= 1e-4 (%d iterations, %d inner steps, "
                     "rel-KKT %.2e), OpenMP build on %d threads" % (info["iters"], info["inner_total"],
                                                                     info["kkt"]["rel_kkt"], used),
           "iters": info["iters"]}
    if not args.cpu_all_only:
        t1, _, info1 = _oracle_solve_timed(inst, 0)
        out["single_thread"] = {"value": t1, "unit": "s", "cores": 1, "iters": info1["iters"]}
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle on the bench's instance, each step one full solve to
    relative KKT <= 1e-4 with the OpenMP build on every host core."""
    if rank != 0:
        return
    import oracle
    oracle.build(omp=True)
    inst = make_instance(args, 0)
    nproc = os.cpu_count() or 1
    vals, used, info = [], 1, None
    for i in range(args.warmup + args.steps):
        t, used, info = _oracle_solve_timed(inst, nproc)
        if i >= args.warmup:
            vals.append(t)
    v = statistics.mean(vals)
    sample = ("each step one full FP64 oracle solve of the bench instance to rel-KKT <= 1e-4 (%d iterations), "
              "OpenMP build on %d threads of %d host cores" % (info["iters"], used, nproc))
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (Philox-seeded)", "impl": "reference",
            "config": {"workload": WORKLOAD, "tol": 1e-4},
            "cpu_baseline": {"kind": "oracle", "cores": used, "sample": sample, "value": v, "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "step_times_s": vals}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-all-only", action="store_true", help="cpu_baseline: skip the single-thread solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="leave the large sparse QP out of the default line")
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--small", action="store_true", help="10x smaller instance (quick checks)")
    ap.add_argument("--workload", default="socp", choices=["socp", "portfolio", "large", "gemm", "lasso", "qcqp", "spmv"])
    ap.add_argument("--ws-train", type=int, default=0, help="portfolio: instances to train the warm start on")
    ap.add_argument("--ws-steps", type=int, default=3000, help="portfolio: warm-start training steps")
    ap.add_argument("--large-n", type=float, default=2e8, help="large: number of variables")
    ap.add_argument("--matrix-bf16", type=int, default=0,
                    help="large: 2 = BF16-stored values of A, A' and P (the BF16-rounded problem is solved)")
    args = ap.parse_args()
    if args.workload != "socp" and args.impl == "ours":
        {"portfolio": run_portfolio, "large": run_large, "gemm": run_gemm, "spmv": run_spmv, "lasso": run_frontend,
         "qcqp": run_frontend}[args.workload](args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group(backend="nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
