#!/usr/bin/env python
"""Benchmark: first-order Magnus intervals per second on the d = 729 transmon chain.

Workload: chain of 6 three-level transmons (d = 729), 6 Gaussian-cosine drives,
2000 Magnus intervals of 16 Gauss-Legendre points over T = 50 ns, full
propagator U(T) = U_1999 ... U_0.  One step = one pass of the whole path on one
GPU: quadrature coefficients, Hbar_n, FP64 norms, exponentials (Taylor +
squaring on the tcgen05 split-precision products), tree product.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is device-timed throughput with inputs resident
in HBM; `e2e` repeats the step through the same C ABI with host buffers
(samples host->device, U device->host inside the timed region).  The CPU oracle
(`--impl reference`, and the `cpu_baseline` sample) runs on the host cores.
Under torchrun each rank evolves its own independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Magnus intervals/sec at dim 729 vs FP64 err; p50/p99 latency, mixed stream"
UNIT = "intervals/s"
WORKLOAD = "transmon_chain_d729_N2000_P16_K6_propagator"
SAMPLE_INTERVALS = 128          # oracle sample (cpu_baseline) and accuracy prefix
# DRAM bytes (read + write) of the split-product launches per flop of algorithmic work they
# count, keyed by (d, digits): the summed ncu DRAM bytes of every product launch of one pass
# over 32 intervals (three power products, three symmetric products, the tree) divided by
# their summed algorithmic work; the bench scales it to the average timed launch by the work
# that launch counts (the pass has the timed step's mix of products per interval).  An entry
# is valid for the kernel build it was captured from only, and is removed when it changes.
GEMM_DRAM_BYTES_PER_FLOP = {(729, 6): 7.720727296e9 / 2.82297207672e11}
REFERENCE_STEP_INTERVALS = 16   # oracle intervals per step of --impl reference
# FP64 and TF32 dense matrix-product peaks of GB300 measured by `python bench.py --peaks`
# (torch.matmul, n = 8192, best of 10, CUDA events); the BF16 peaks come from MEASURED_PEAKS.json
FP64_TFLOPS_MEASURED = 1.10
TF32_TFLOPS_MEASURED = 1024.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["split", "fp64"], default="split")
    ap.add_argument("--slices", type=int, default=6)
    ap.add_argument("--stage-k", type=int, default=32, choices=[16, 32, 64],
                    help="K per pipeline stage of the split product (mg_ctx_set_stage_k)")
    ap.add_argument("--digit-pairs", type=int, default=None, choices=[0, 1, 2],
                    help="paired digit layout of the split product (mg_ctx_set_digit_pairs)")
    ap.add_argument("--cta-pairs", type=int, default=None, choices=[0, 1],
                    help="split products on CTA pairs (mg_ctx_set_cta_pairs)")
    ap.add_argument("--workspace-gib", type=float, default=None,
                    help="device workspace limit of the context (mg_ctx_set_workspace_limit): by default 64 GiB "
                         "for the headline (491 intervals per chunk at d = 729; 4525 vs 4428 intervals/s with "
                         "the library's 16 GiB, 123 per chunk), the library default elsewhere")
    ap.add_argument("--no-structure", action="store_true",
                    help="full split products even for real operators (mg_ctx_set_structure 0)")
    ap.add_argument("--tolerance", type=float, default=1e-6,
                    help="max-abs tolerance the headline plan is tuned for (mg_plan_autotune)")
    ap.add_argument("--no-tune", action="store_true",
                    help="headline: keep --precision/--slices instead of tuning for --tolerance")
    ap.add_argument("--taylor-target", type=float, default=0.0,
                    help="with --no-tune: the headline plan's Taylor truncation target (mg_plan_set_taylor_target)")
    ap.add_argument("--intervals", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="default line: skip the served-stream measurement (p50/p99 on a prefix of the stream)")
    ap.add_argument("--serve-requests", type=int, default=64,
                    help="default line: requests of the served stream's prefix")
    ap.add_argument("--config", type=int, default=1,
                    help="1: d = 729 chain (headline); 0: d = 30 transmon-resonator state, FP64; "
                         "2: 512 uneven instances batched; 3: d = 4096 all-to-all, tree product; "
                         "4: served request stream (p50/p99)")
    ap.add_argument("--requests", type=int, default=48, help="config 4: requests taken from the stream")
    ap.add_argument("--rate", type=float, default=200.0,
                    help="config 4: offered request rate (the Poisson stream's arrival times are stretched "
                         "from 200/s to this rate; the requests themselves are unchanged)")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 and TF32 matrix-product peaks with torch.matmul (CUDA events, best "
                         "of 10) and print them")
    ap.add_argument("--shard", action="store_true",
                    help="d = 729 chain: one job's 2000 intervals shared by the ranks (each rank's ranges by "
                         "mg_evolve, one NCCL all-gather of the partials, the ordered product by mg_cgemm) "
                         "instead of one replica per rank")
    ap.add_argument("--virtual", type=int, default=1, help="--shard: interval ranges per rank")
    ap.add_argument("--tune", action="store_true",
                    help="run the autotuner (mg_plan_autotune) on the d = 30, d = 729 and a 512-batch instance "
                         "workload and print every measured candidate")
    ap.add_argument("--graph", action="store_true",
                    help="config 2: the batch captured once in a CUDA graph (mg_batch_graph_*) and replayed "
                         "every step")
    ap.add_argument("--action", action="store_true",
                    help="configs 0, 2, 3: state outputs by the action of exp(-i Hbar_n) on psi (sparse "
                         "operators, FP64); config 3 then evolves the state |0> instead of the full propagator; "
                         "config 4: state requests are flagged for the action path (the server takes it "
                         "from d = 256)")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local



def tune_plan(M, torch, stream, plan, output, tolerance, set_controls):
    """mg_plan_autotune for `tolerance` before the timed region.  When no measured
    candidate qualifies (its error estimate times the safety factor 4 above the
    tolerance) the plan keeps its configuration and the line says so."""
    info = {"tolerance": tolerance, "safety_factor": 4}
    t0 = time.perf_counter()
    try:
        with torch.cuda.stream(stream):
            set_controls()
            info["chosen"] = plan.autotune(output, tolerance, None)
    except M.MagnusError as e:
        if e.code != M.MG_EUNSUPPORTED:
            raise
        info["chosen"] = None
        info["kept"] = "no candidate's estimated error x 4 met the tolerance; the plan keeps its configuration"
    info["seconds"] = time.perf_counter() - t0
    return info


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max([num(r[3]) for r in rows if num(r[3]) is not None] or [0.0])}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import workloads as W
    from paper_2411_09982_gb300 import build as B
    from paper_2411_09982_gb300 import magnus as M

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    B.build()
    M.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    ctx = M.Context(local, stream)
    ctx.set_stage_k(args.stage_k)
    if args.digit_pairs is not None:
        ctx.set_digit_pairs(args.digit_pairs)
    if args.cta_pairs is not None:
        ctx.set_cta_pairs(args.cta_pairs)
    if args.no_structure:
        ctx.set_structure(False)
    if args.workspace_gib is None:
        args.workspace_gib = 64.0
    ctx.set_workspace_limit(int(args.workspace_gib * (1 << 30)))
    prec = M.MG_PREC_SPLIT if args.precision == "split" else M.MG_PREC_FP64
    N = args.intervals

    wl = W.config(1, seed=1 + rank)
    samples_np, w = M.node_samples(wl, N)
    H0 = torch.from_numpy(wl.H0).to(dev)
    Hk = torch.from_numpy(wl.Hk).to(dev)
    samples = torch.from_numpy(samples_np).to(dev)
    samples_host = torch.from_numpy(samples_np).pin_memory()
    out = torch.empty((wl.d, wl.d), dtype=torch.complex128, device=dev)
    out_host = torch.empty((wl.d, wl.d), dtype=torch.complex128).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MiB > L2
    plan = M.Plan(ctx, H0, Hk, prec, args.slices)
    slices = args.slices
    tuning = None
    if args.no_tune and args.taylor_target:
        plan.set_taylor_target(args.taylor_target)
    if prec == M.MG_PREC_SPLIT and not args.no_tune:
        # configuration (digits, Taylor scheme and truncation target, hence squarings) chosen
        # by the library's autotuner for the stated tolerance, measured before the timed region
        tuning = tune_plan(M, torch, stream, plan, M.MG_OUT_PROPAGATOR, args.tolerance,
                           lambda: plan.set_controls(N, wl.P, wl.t0, wl.dt, w, samples))
        if tuning.get("chosen"):
            prec = tuning["chosen"]["precision"]
            slices = tuning["chosen"]["slices"] if prec == M.MG_PREC_SPLIT else None

    def configure(p):
        """The headline plan's configuration on another plan of the same operators."""
        if tuning is not None and tuning.get("chosen"):
            p.set_taylor(tuning["chosen"]["taylor"])
            p.set_taylor_target(tuning["chosen"]["taylor_target"])
        elif args.no_tune and args.taylor_target:
            p.set_taylor_target(args.taylor_target)

    def step():
        plan.set_controls(N, wl.P, wl.t0, wl.dt, w, samples)
        plan.evolve(M.MG_OUT_PROPAGATOR, None, out, 0, report=False)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
        stream.synchronize()

        # ---- timed region: K steps, L2 flushed before each, CUDA events on the library's stream
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        launches0 = M.mg_kernel_launch_count()
        ctx.gemm_stats(reset=True)
        ctx.enable_gemm_timing(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        stream.synchronize()
        ctx.enable_gemm_timing(False)
        gstats = ctx.gemm_stats(reset=True)
        launches = M.mg_kernel_launch_count() - launches0
        torch.cuda.synchronize()
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_ms = sum(step_ms)
        if ws > 1:
            t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_ms = float(t.item())
            torch.distributed.barrier()

        # ---- end to end through the C ABI with host buffers
        e2e_steps = args.e2e_steps or args.steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.set_controls(N, wl.P, wl.t0, wl.dt, w, samples_host)
            plan.evolve(M.MG_OUT_PROPAGATOR, None, out_host, 0, host=True, report=False)
        stream.synchronize()
        e2e_s = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(t.item())

    value = ws * N * args.steps / (total_ms / 1000.0)
    e2e_value = ws * N * e2e_steps / e2e_s

    result = None
    if rank == 0:
        peaks, peak_src = measured_peaks()
        # dominant kernel: the matrix-product launches (split GEMM or FP64 GEMM)
        per_launch_ms = gstats["ms"] / max(1, gstats["launches"])
        per_launch_flops = gstats["flops"] / max(1, gstats["launches"])
        achieved = per_launch_flops / (per_launch_ms * 1e-3) / 1e12
        if prec == M.MG_PREC_SPLIT:
            peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
            pairs = slices * (slices + 1) // 2
            per_flop = GEMM_DRAM_BYTES_PER_FLOP.get((wl.d, slices)) if not args.no_structure else None
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "traffic": per_flop * per_launch_flops if per_flop else None,
                    "traffic_note": "bytes per average launch: ncu DRAM bytes per counted flop of one "
                                    "32-interval pass, times the launch's counted work",
                    "kernel": "split_gemm_kernel",
                    "peak_source": f"bf16 dense sustained, {peak_src}",
                    "note": f"achieved counts algorithmic work: 8 d^3 flops per general complex product, "
                            f"a quarter of that where both operands have a zero part (powers of X with "
                            f"real operators), and d (d + 1) / 2 of the d^2 outputs of a symmetric "
                            f"result; the tensor pipe issues {pairs} BF16 digit-pair products per such "
                            f"flop"}
        else:
            fp64_peak = FP64_TFLOPS_MEASURED
            roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": None, "kernel": "cgemm_f64_kernel",
                    "peak_source": "FP64 torch.matmul, measured (bench.py --peaks)"}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": (f"bf16 digits x{slices} (fp32 accumulate) + f64" if prec == M.MG_PREC_SPLIT else "f64"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "d": wl.d, "intervals": N, "quadrature_points": wl.P,
                       "controls": wl.K, "output": "full propagator",
                       "precision": "split" if prec == M.MG_PREC_SPLIT else "fp64",
                       "slices": slices if prec == M.MG_PREC_SPLIT else None,
                       "tuning": tuning,
                       "taylor_target": args.taylor_target if args.no_tune and args.taylor_target else None,
                       "l2": "256 MiB buffer written before every timed step",
                       "workspace_gib": args.workspace_gib,
                       "parallelism": "independent replica per GPU"},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(samples_host.numel() * 8),
                    "d2h_bytes_per_step": int(out_host.numel() * 16)},
            "clocks": clk,
            "gpu_launches": int(launches),
            "gemm_launches_timed": int(gstats["launches"]),
        }
        # accuracy vs the FP64 oracle and the CPU baseline on the same prefix
        if not args.no_cpu_baseline:
            import oracle
            n_s = min(SAMPLE_INTERVALS, N)
            cores = len(os.sched_getaffinity(0))
            t0 = time.perf_counter()
            ref = oracle.evolve_workload(wl, n_intervals=n_s)
            cpu_s = time.perf_counter() - t0
            with torch.cuda.stream(stream):
                pre = M.Plan(ctx, H0, Hk, prec, slices if prec == M.MG_PREC_SPLIT else args.slices)
                configure(pre)
                pre.set_controls(n_s, wl.P, wl.t0, wl.dt, w, samples[:n_s].contiguous())
                pre.evolve(M.MG_OUT_PROPAGATOR, None, out, 0, report=False)
                stream.synchronize()
                err = float(np.abs(out.cpu().numpy() - ref).max())
                pre.close()
            result["cpu_baseline"] = {"value": n_s / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                                      "sample": f"first {n_s} of the {N} intervals of the same workload "
                                                f"(numpy eigh exponentials, sequential products)"}
            result["accuracy"] = {"max_abs_err_vs_fp64_oracle": err, "intervals_compared": n_s,
                                  "tolerance": 1e-6 if prec == M.MG_PREC_SPLIT else 1e-11}
        # U(T) of the last timed step over all N intervals against the oracle's sampled entries
        # (tests/golden, written by a script that runs only the CPU oracle)
        gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                            "chain_d729_N2000_propagator.json")
        if os.path.exists(gold) and N == 2000 and rank == 0:
            with open(gold) as f:
                g = json.load(f)
            e = np.array(g["entries"])
            with torch.cuda.stream(stream):
                plan.set_controls(N, wl.P, wl.t0, wl.dt, w, samples)
                plan.evolve(M.MG_OUT_PROPAGATOR, None, out, 0, report=False)
                stream.synchronize()
            U = out.cpu().numpy()
            err_all = float(np.abs(U[e[:, 0].astype(int), e[:, 1].astype(int)] - (e[:, 2] + 1j * e[:, 3])).max())
            result.setdefault("accuracy", {})["max_abs_err_all_intervals"] = err_all
            result["accuracy"]["all_intervals_compared"] = f"{len(e)} sampled entries of U(T) after all {N}"
    plan.close()
    if result is not None and ws == 1 and not args.no_serving:
        # the served stream beside the headline: the first requests of the Poisson(200/s)
        # mixed stream at the stated rate (an overload) and at half the capacity that run
        # measured; state requests of d >= 256 on the action path, the rest split (6 digits, 7 above d = 1024).
        # A failure here is reported in the line, not raised: the headline stands.
        try:
            with torch.cuda.stream(stream):
                over = serve_prefix(M, W, torch, ctx, dev, args.serve_requests, 200.0, args.slices, True)
                cap = over["requests"] / over["makespan_s"]
                half = serve_prefix(M, W, torch, ctx, dev, args.serve_requests, 0.5 * cap, args.slices, True)
            keys = ("offered_rate_per_s", "latency_ms", "intervals_per_s", "completed", "failed", "makespan_s",
                    "arrival_span_s", "admission_retries", "clocks")
            result["serving"] = {
                "workload": f"first {over['requests']} requests of the Poisson(200/s) mixed stream "
                            f"(d up to {over['d_max']}, {over['intervals_total']} intervals, state or full U)",
                "state_requests": "action path (FP64) from d = 256; the rest split, 6 digits (7 above d = 1024)",
                "at_stated_rate": {k: over[k] for k in keys},
                "capacity_requests_per_s": cap,
                "at_half_capacity": {k: half[k] for k in keys},
            }
            if not args.no_cpu_baseline:
                import oracle
                acc, _ = serve_accuracy(oracle, np, half, len(os.sched_getaffinity(0)))
                result["serving"]["accuracy"] = acc
        except Exception as e:   # noqa: BLE001
            result["serving"] = {"error": f"{type(e).__name__}: {e}"}
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)


# ----------------------------------------------------------------------------
# one job shared by the ranks (interval-range sharding)
# ----------------------------------------------------------------------------
def run_shard(args):
    import torch
    import torch.distributed as dist

    import workloads as W
    from paper_2411_09982_gb300 import build as B
    from paper_2411_09982_gb300 import magnus as M
    from paper_2411_09982_gb300 import shard

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if not dist.is_initialized():
        if ws > 1:
            dist.init_process_group("nccl", init_method="env://")
        else:
            import socket
            sk = socket.socket()
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
            sk.close()
            dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    B.build()
    M.load()
    dev = torch.device("cuda", local)
    ctx = M.Context(local)
    wl = W.config(1)   # the same job on every rank
    N = args.intervals
    sn, w = M.node_samples(wl, N)
    S = torch.from_numpy(sn).to(dev)
    H0, Hk = torch.from_numpy(wl.H0).to(dev), torch.from_numpy(wl.Hk).to(dev)
    prec = M.MG_PREC_SPLIT if args.precision == "split" else M.MG_PREC_FP64
    plan = M.Plan(ctx, H0, Hk, prec, args.slices)

    def step():
        return shard.evolve_propagator_sharded(ctx, H0, Hk, S, N, wl.P, wl.t0, wl.dt, w, prec, args.slices,
                                               virtual=args.virtual, plan=plan)

    for _ in range(max(3, args.warmup)):
        step()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = step()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    el = shard.max_over_ranks(el, device=dev)
    if rank == 0:
        print(json.dumps({"metric": METRIC + " (one job shared by the ranks)", "value": N * args.steps / el,
                          "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup),
                          "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True, "scaling": "strong",
                          "vs_baseline": None, "data": "synthetic",
                          "config": {"workload": WORKLOAD, "intervals": N, "ranges": ws * args.virtual,
                                     "precision": args.precision,
                                     "exchange": "NCCL all-gather of the d x d partials, product by mg_cgemm"},
                          "unitarity_check": float((U.conj().T @ U - torch.eye(wl.d, device=dev,
                                                                               dtype=U.dtype)).abs().max())}),
              flush=True)
    plan.close()
    ctx.close()
    dist.destroy_process_group()


# ----------------------------------------------------------------------------
# the served stream (config 4): a prefix of the Poisson request stream
# ----------------------------------------------------------------------------
def serve_prefix(M, W, torch, ctx, dev, requests, rate, slices, action):
    """Submit the first `requests` requests of the 200/s Poisson stream to one server at their
    arrival times stretched to `rate` requests/s (the requests themselves unchanged) and wait
    for all.  State requests take the action path from d = 256 when `action`."""
    stretch = 200.0 / rate
    stream_spec = [(arr * stretch, sp) for arr, sp in W.serving_stream()[:requests]]
    built = [W.serving_job(sp) for _, sp in stream_spec]
    inputs = []
    for wl in built:
        sn, w = M.node_samples(wl)
        inputs.append((torch.from_numpy(wl.H0).to(dev), torch.from_numpy(wl.Hk).to(dev),
                       torch.from_numpy(sn).to(dev), w,
                       torch.from_numpy(wl.psi0).to(dev) if wl.psi0 is not None else None,
                       torch.empty(wl.d if wl.psi0 is not None else (wl.d, wl.d), dtype=torch.complex128,
                                   device=dev)))
    torch.cuda.synchronize()
    srv = M.Server(ctx, mem_budget_bytes=64 << 30, quantum_intervals=256)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    t_start = time.perf_counter()
    ids, rejected, flagged = [], 0, []
    for (arr, sp), wl, (H0, Hk, S, w, inp, o) in zip(stream_spec, built, inputs):
        now = time.perf_counter() - t_start
        if arr > now:
            time.sleep(arr - now)
        kind = M.MG_OUT_STATE if inp is not None else M.MG_OUT_PROPAGATOR
        act = action and kind == M.MG_OUT_STATE
        while True:
            # digits carrying 42 bits at the request's d (one more above d = 1024, where beta = 6)
            sl = max(slices, M.mg_split_digits(wl.d, 7 * slices)[1])
            jid = srv.submit(H0, Hk, wl.N, wl.P, wl.t0, wl.dt, w, S, kind, inp, o, M.MG_PREC_SPLIT, sl,
                             action=act)
            if jid is not None:
                break
            rejected += 1
            time.sleep(0.01)
        ids.append(jid)
        flagged.append(act and wl.d >= 256)
    reps = [srv.wait(j, 3600.0) for j in ids]
    wall = time.perf_counter() - t_start
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    failed = sum(1 for r in reps if r is None or r["status"] != 0)
    lat = sorted(r["latency_ms"] for r in reps if r is not None)
    intervals = sum(wl.N for wl in built)
    return {"requests": len(ids), "offered_rate_per_s": rate, "arrival_span_s": stream_spec[-1][0],
            "d_max": max(wl.d for wl in built), "intervals_total": intervals, "makespan_s": wall,
            "intervals_per_s": intervals / wall, "completed": st["completed"], "failed": failed,
            "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "max": lat[-1]},
            "admission_retries": rejected, "clocks": clk, "_built": built, "_inputs": inputs, "_fp64": flagged}


def serve_accuracy(oracle, np, res, cores, budget_s=15.0, at_least=8):
    """The oracle on the cheapest served requests (by d^3 N), at least `at_least` of them and
    more while the host budget lasts, against the served results."""
    built, inputs, fp64 = res["_built"], res["_inputs"], res["_fp64"]
    order = sorted(range(len(built)), key=lambda q: built[q].d ** 3 * built[q].N)
    t0 = time.perf_counter()
    done_n, errs = 0, {"split": [], "fp64_action": []}
    for k, q in enumerate(order):
        if k >= at_least and time.perf_counter() - t0 > budget_s:
            break
        ref = oracle.evolve_workload(built[q])
        errs["fp64_action" if fp64[q] else "split"].append(float(np.abs(inputs[q][5].cpu().numpy() - ref).max()))
        done_n += built[q].N
    cpu_s = time.perf_counter() - t0
    n = sum(len(v) for v in errs.values())
    acc = {"requests_compared": n,
           "max_abs_err_vs_fp64_oracle_split": max(errs["split"]) if errs["split"] else None,
           "max_abs_err_vs_fp64_oracle_action": max(errs["fp64_action"]) if errs["fp64_action"] else None,
           "tolerance": {"split": 1e-6, "action (FP64)": 1e-11}}
    cpu = {"value": done_n / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"the {n} cheapest requests of the stream (by d^3 N)"}
    return acc, cpu


# ----------------------------------------------------------------------------
# the other workloads (one GPU; not the default line)
# ----------------------------------------------------------------------------
def run_config(args):
    import numpy as np
    import torch

    import oracle
    import workloads as W
    from paper_2411_09982_gb300 import build as B
    from paper_2411_09982_gb300 import magnus as M

    B.build()
    M.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    ctx = M.Context(0, stream)
    ctx.set_stage_k(args.stage_k)
    if args.digit_pairs is not None:
        ctx.set_digit_pairs(args.digit_pairs)
    if args.cta_pairs is not None:
        ctx.set_cta_pairs(args.cta_pairs)
    if args.no_structure:
        ctx.set_structure(False)
    if args.workspace_gib:
        ctx.set_workspace_limit(int(args.workspace_gib * (1 << 30)))
    cores = len(os.sched_getaffinity(0))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    warm = max(3, args.warmup)
    out_line = {"metric": None, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": warm,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}

    def timed(step, steps):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                step()
            stream.synchronize()
            clocks = ClockSampler(0)
            clocks.start()
            l0 = M.mg_kernel_launch_count()
            ctx.gemm_stats(reset=True)
            ctx.enable_gemm_timing(True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for i in range(steps):
                flush.zero_()
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            stream.synchronize()
            ctx.enable_gemm_timing(False)
            g = ctx.gemm_stats(reset=True)
            clk = clocks.stop()
        return sum(a.elapsed_time(b) for a, b in ev), g, clk, M.mg_kernel_launch_count() - l0

    def gemm_roof(g, pairs, clk=None):
        if not g["launches"]:
            return None
        ach = g["flops"] / (g["ms"] * 1e-3) / 1e12
        peaks, src = measured_peaks()
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        p64 = FP64_TFLOPS_MEASURED
        return {"bound": "tensor" if pairs else "alu", "achieved": ach, "peak": peak if pairs else p64,
                "unit": "TFLOP/s", "frac": ach / (peak if pairs else p64), "traffic": None,
                "peak_source": f"bf16 dense sustained, {src}" if pairs else
                "FP64 torch.matmul, measured (bench.py --peaks)"}

    aflag = M.MG_FLAG_STATE_ACTION if args.action else 0
    if args.config in (0, 3):
        wl = W.config(args.config)
        if args.action and wl.psi0 is None:
            wl.psi0 = W.basis_state(wl.d, 0)
            wl.name += "_state"
        prec = M.MG_PREC_FP64 if args.config == 0 or args.action else M.MG_PREC_SPLIT
        reorth = 64 if args.config == 3 and not args.action else 0
        samples_np, w = M.node_samples(wl)
        samples = torch.from_numpy(samples_np).to(dev)
        # d = 4096 needs 7 digits for 1e-6 over its 500 intervals (beta = 6: six carry 36 bits)
        base_slices = 7 if args.config == 3 and args.slices == 6 else args.slices
        plan = M.Plan(ctx, torch.from_numpy(wl.H0).to(dev), torch.from_numpy(wl.Hk).to(dev), prec, base_slices,
                      aflag)
        state = wl.psi0 is not None
        inp = torch.from_numpy(wl.psi0).to(dev) if state else None
        out = torch.empty(wl.d if state else (wl.d, wl.d), dtype=torch.complex128, device=dev)
        slices = base_slices
        tuning = None
        if prec == M.MG_PREC_SPLIT and not args.no_tune:
            # digits, Taylor scheme and truncation target chosen by the autotuner for the tolerance
            tuning = tune_plan(M, torch, stream, plan, M.MG_OUT_STATE if state else M.MG_OUT_PROPAGATOR,
                               args.tolerance, lambda: plan.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, samples))
            if tuning.get("chosen"):
                prec = tuning["chosen"]["precision"]
                slices = tuning["chosen"]["slices"] if prec == M.MG_PREC_SPLIT else base_slices

        def step():
            plan.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, samples)
            plan.evolve(M.MG_OUT_STATE if state else M.MG_OUT_PROPAGATOR, inp, out, reorth, report=False)

        ms, g, clk, launches = timed(step, args.steps)
        out_line.update(metric=f"Magnus intervals/sec, {wl.name}", value=wl.N * args.steps / (ms / 1e3),
                        ms_per_step=ms / args.steps, dtype="f64" if prec == M.MG_PREC_FP64 else
                        f"bf16 digits x{slices} (fp32 accumulate) + f64",
                        config={"workload": wl.name, "d": wl.d, "intervals": wl.N, "quadrature_points": wl.P,
                                "controls": wl.K, "output": "state" if state else "full propagator",
                                "method": "action (Chebyshev, sparse)" if args.action else "interval propagators",
                                "reorth_every": reorth, "tuning": tuning,
                                "l2": "256 MiB buffer written before every timed step"},
                        roofline=gemm_roof(g, 0 if prec == M.MG_PREC_FP64 else slices * (slices + 1) // 2, clk),
                        clocks=clk, gpu_launches=int(launches))
        gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                            "alltoall_d4096_N500_first130_propagator.json")
        if args.config == 3 and not state and os.path.exists(gold):
            # the first intervals (two re-orthonormalisation boundaries) against the oracle's sampled entries
            with open(gold) as f:
                gd = json.load(f)
            n_g = gd["workload"]["intervals_applied"]
            e = np.array(gd["entries"])
            with torch.cuda.stream(stream):
                plan.set_controls(n_g, wl.P, wl.t0, wl.dt, w, samples[:n_g].contiguous())
                plan.evolve(M.MG_OUT_PROPAGATOR, None, out, reorth, report=False)
                stream.synchronize()
            U = out.cpu().numpy()
            out_line["accuracy"] = {
                "max_abs_err_vs_fp64_oracle": float(np.abs(U[e[:, 0].astype(int), e[:, 1].astype(int)]
                                                           - (e[:, 2] + 1j * e[:, 3])).max()),
                "intervals_compared": n_g, "compared": f"{len(e)} sampled entries of U after {n_g} intervals",
                "tolerance": args.tolerance}
        if args.action:
            rep = plan.evolve(M.MG_OUT_STATE, inp, out, 0)
            out_line["action"] = {k: rep[k] for k in ("sparse_matvecs", "sparse_nnz", "max_squarings",
                                                      "taylor_degree", "max_norm1", "action_ctas")}
        if not args.no_cpu_baseline:
            n_s = 128 if args.config == 0 else 1
            t0 = time.perf_counter()
            ref = oracle.evolve_workload(wl, n_intervals=n_s)
            cpu_s = time.perf_counter() - t0
            out_line["cpu_baseline"] = {"value": n_s / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                                        "sample": f"first {n_s} intervals of the workload"}
            if args.config == 0:
                full = oracle.evolve_workload(wl)
                with torch.cuda.stream(stream):
                    step()
                    stream.synchronize()
                out_line["accuracy"] = {"max_abs_err_vs_fp64_oracle": float(np.abs(out.cpu().numpy() - full).max()),
                                        "intervals_compared": wl.N, "tolerance": 1e-11}
        plan.close()
    elif args.config == 2:
        jobs = W.uneven_batch()
        plans, kinds, ins, outs, samp = [], [], [], [], []
        for wl in jobs:
            sn, w = M.node_samples(wl)
            st = torch.from_numpy(sn).to(dev)
            p = M.Plan(ctx, torch.from_numpy(wl.H0).to(dev), torch.from_numpy(wl.Hk).to(dev),
                       M.MG_PREC_FP64 if args.action else M.MG_PREC_SPLIT, args.slices, aflag)
            plans.append(p)
            samp.append((st, w))
            kinds.append(M.MG_OUT_STATE)
            ins.append(torch.from_numpy(wl.psi0).to(dev))
            outs.append(torch.empty(wl.d, dtype=torch.complex128, device=dev))
        total = sum(wl.N for wl in jobs)
        graph = None
        if args.graph:
            for p, wl, (st, w) in zip(plans, jobs, samp):
                p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, st)
            with torch.cuda.stream(stream):
                graph = M.BatchGraph(ctx, plans, kinds, ins, outs)

        def step():
            for p, wl, (st, w) in zip(plans, jobs, samp):
                p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, st)
            if graph is not None:
                status = graph.launch()
            else:
                status = M.mg_evolve_batch(ctx, plans, kinds, ins, outs)
            assert status == [0] * len(jobs), "a job of the batch failed"

        ms, g, clk, launches = timed(step, args.steps)
        ds = sorted(wl.d for wl in jobs)
        out_line.update(metric="Magnus intervals/sec, 512 uneven transmon-resonator instances (batched)",
                        value=total * args.steps / (ms / 1e3), ms_per_step=ms / args.steps,
                        dtype="f64" if args.action else f"bf16 digits x{args.slices} (fp32 accumulate) + f64",
                        config={"workload": "uneven_batch_512", "jobs": len(jobs), "intervals_total": total,
                                "d_min": ds[0], "d_median": ds[len(ds) // 2], "d_max": ds[-1],
                                "output": "state",
                                "method": "action (Chebyshev, sparse)" if args.action else "interval propagators",
                                "issue": "one captured CUDA graph per step" if graph is not None
                                else "stream launches, no host synchronisation between chunks",
                                "l2": "256 MiB buffer written before every timed step"},
                        roofline=gemm_roof(g, 0 if args.action else args.slices * (args.slices + 1) // 2, clk),
                        clocks=clk, gpu_launches=int(launches),
                        launches_per_step=int(launches) / args.steps)
        if graph is not None:
            out_line["graph"] = graph.stats()
        if not args.no_cpu_baseline:
            sample = jobs[:3]
            t0 = time.perf_counter()
            refs = [oracle.evolve_workload(wl) for wl in sample]
            cpu_s = time.perf_counter() - t0
            out_line["cpu_baseline"] = {"value": sum(wl.N for wl in sample) / cpu_s, "unit": UNIT, "cores": cores,
                                        "kind": "oracle", "sample": "the first 3 instances of the batch"}
            err = max(float(np.abs(o.cpu().numpy() - r).max()) for o, r in zip(outs[:3], refs))
            out_line["accuracy"] = {"max_abs_err_vs_fp64_oracle": err, "jobs_compared": 3,
                                    "tolerance": 1e-11 if args.action else 1e-6}
        if graph is not None:
            graph.close()
        for p in plans:
            p.close()
    elif args.config == 4:
        res = serve_prefix(M, W, torch, ctx, dev, args.requests, args.rate, args.slices, args.action)
        out_line.update(metric="served Magnus stream: intervals/sec with p50/p99 request latency",
                        value=res["intervals_per_s"], ms_per_step=None, steps=1, warmup=0,
                        dtype=f"bf16 digits x{args.slices} (fp32 accumulate) + f64",
                        config={"workload": "poisson_200_per_s_mixed_d32_2048", "requests": res["requests"],
                                "offered_rate_per_s": args.rate, "arrival_span_s": res["arrival_span_s"],
                                "d_max": res["d_max"], "intervals_total": res["intervals_total"],
                                "quantum_intervals": 256,
                                "state_requests": "action path (FP64) from d = 256" if args.action else "split path"},
                        latency_ms=res["latency_ms"], admission_retries=res["admission_retries"],
                        clocks=res["clocks"])
        if not args.no_cpu_baseline:
            acc, cpu = serve_accuracy(oracle, np, res, cores)
            out_line["cpu_baseline"] = cpu
            out_line["accuracy"] = acc
    ctx.close()
    print(json.dumps(out_line), flush=True)


# ----------------------------------------------------------------------------
# FP64 and TF32 peaks (torch.matmul), for the fractions of the FP64 and TF32 paths
# ----------------------------------------------------------------------------
def run_peaks(args):
    import torch
    out = {}
    for name, dtype, tf32, n in (("fp64", torch.float64, False, 8192), ("tf32", torch.float32, True, 8192),
                                 ("bf16", torch.bfloat16, False, 8192)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(3):
            torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[f"{name}_tflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    out["how"] = "torch.matmul n = 8192 (2 n^3 flops), best of 10 after 3 warm-up, CUDA events"
    out["gpu"] = torch.cuda.get_device_name(0)
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------
# the autotuner's measured tables
# ----------------------------------------------------------------------------
def run_tune(args):
    import tempfile

    import torch

    import workloads as W
    from paper_2411_09982_gb300 import build as B
    from paper_2411_09982_gb300 import magnus as M

    B.build()
    M.load()
    ctx = M.Context(0, torch.cuda.Stream())
    cases = [(W.config(0), M.MG_OUT_STATE, 1e-11), (W.config(0), M.MG_OUT_STATE, 1e-6),
             (W.config(1), M.MG_OUT_PROPAGATOR, 1e-6), (W.config(1), M.MG_OUT_PROPAGATOR, 1e-4),
             (W.uneven_batch()[0], M.MG_OUT_STATE, 1e-6)]
    names = {(0, 0): "fp64", (1, 0): "split"}
    for wl, output, tol in cases:
        fd, path = tempfile.mkstemp(suffix=".txt")
        os.close(fd)
        os.unlink(path)
        sn, w = M.node_samples(wl)
        plan = M.Plan(ctx, torch.from_numpy(wl.H0).cuda(), torch.from_numpy(wl.Hk).cuda(), M.MG_PREC_SPLIT, 6)
        plan.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, torch.from_numpy(sn).cuda())
        chosen = plan.autotune(output, tol, path)
        key, sel, ents = open(path).read().strip().split("\t")
        table = []
        for e in ents.split(";"):
            p, s_, t, a, err, us, *tu = e.split()
            table.append({"path": "action" if int(a) else names[(int(p), 0)], "digits": int(s_) or None,
                          "taylor": "ps" if int(t) else "deg18", "error_est": float(err),
                          "us_per_interval": float(us), "taylor_target": float(tu[0]) if tu else 0.0})
        print(json.dumps({"workload": wl.name, "d": wl.d, "N": wl.N, "output": "state" if output == 0 else "U",
                          "tolerance": tol, "key": key, "selected": int(sel), "chosen": chosen,
                          "candidates": table}), flush=True)
        plan.close()
        os.unlink(path)
    ctx.close()


# ----------------------------------------------------------------------------
# reference arm: the CPU FP64 oracle, timed on the host cores (rank 0 only)
# ----------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    import workloads as W
    wl = W.config(1, seed=1)
    n = REFERENCE_STEP_INTERVALS
    cores = len(os.sched_getaffinity(0))
    for _ in range(max(3, args.warmup) if args.warmup else 0):
        oracle.evolve_workload(wl, n_intervals=2)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.evolve_workload(wl, n_intervals=n)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * args.steps / total
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "d": wl.d, "intervals": args.intervals, "quadrature_points": wl.P,
                   "controls": wl.K, "output": "full propagator"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} intervals of the workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.tune:
        run_tune(a)
    elif a.shard:
        run_shard(a)
    elif a.peaks:
        run_peaks(a)
    elif a.config != 1:
        run_config(a)
    else:
        run_ours(a)
