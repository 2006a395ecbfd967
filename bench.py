#!/usr/bin/env python
"""Benchmark of the wall-corrected RPY pair kernel (blob-pair interactions/s)
and of the mobility solves built on it (solves/s, p50/p99 latency).

Workload of the headline: the wall-RPY mobility product u = M f for N = 65,536
free blobs, a = 0.5, x, y ~ U[0, 400], z ~ U[a, 3a], f ~ N(0, 1) (seeded,
synthetic).  One step = one mb_mobility_matvec call (FP32 pair kernel with
hi/lo positions and Kahan-compensated accumulation) on inputs already in HBM;
the L2 is flushed (256 MB write) before every timed step.  Pairs per step = N^2
(self pairs included).

Also reported on the same line:
  e2e          the same metric through the C ABI with host buffers (pinned):
               host->device copies of r and f and the device->host copy of u
               inside the timed region of every step
  roofline     the pair kernel against the FP32 FMA rate measured in this run
               (mb_measure_fma_rate), with the method's flops per ordered pair
               (Eq. RPYTensor plus the wall correction, counted as written)
  cpu_baseline the FP64 oracle on this host's cores, on the 4,096 sampled
               targets of the workload
  matvec_err   the FP32 product against the oracle on those 4,096 targets
               (relative L2 bound 1e-5: the line fails above it)
  matvec_fp64, matvec_df64   the product in FP64 and in double-float, each
               timed and compared with the oracle on the same targets
  solve, solve_fp64   mobility solves of 8 x 42-blob shells (solves/s, p50/p99)
  monolayer    the 4,096 x 162-blob sedimented monolayer solve (mixed, 1e-8)
  batch        256 independent mixed suspensions solved together
  serve        the Poisson serving stream: saturated at 200 req/s, then at
               0.8 x the measured capacity (p50/p99, served/offered, queue)

--impl reference times the FP64 oracle (the reference arm of this repo) on
this host's cores on the same workload, a bounded sample of targets per step.
Multi-GPU: `--gpus N` under torchrun runs N independent replicas (the path is
not sharded here); value = pairs of all ranks / slowest rank's time.  The
solve sections run at N = 1 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 65536
# The method's arithmetic per ordered blob pair, counted from the formulas as
# written (multiplies and adds separately, rsqrt as one; the rare overlap
# branch not counted): the free RPY tensor of Eq. RPYTensor applied to f_j
# (29) and the wall correction with the accumulation into u_i (79).  The FP32
# kernel adds 9 for the separation of its hi/lo positions, a device of its
# precision rather than work of the method, so it is not counted.
FLOPS_PER_PAIR = 108
FLOPS_BASIS = ("Eq. RPYTensor far branch applied to f_j (29) + wall correction and "
               "accumulation (79), as written; the FP32 kernel's hi/lo separation (9) "
               "not counted")
SM_MAX_MHZ = 2070.0
ORACLE_ROWS = 4096  # the workload's oracle subsample of targets
MATVEC_TOL = 1e-5
KERNEL_NAMES = {0: "pair_f32_kernel<wall> (scalar, 1 target/thread)",
                1: "pair_f32x2_kernel<wall,1> (packed f32x2, 2 targets/thread)",
                2: "pair_f32x2_kernel<wall,2> (packed f32x2, 4 targets/thread)",
                3: "pair_sym_kernel<wall> (symmetric packed f32x2, each pair once for both blobs)",
                4: "pair_f32x2_kernel<wall,1,32> (packed f32x2, 32-thread CTAs, small problems)"}
WORKLOAD = "wall-RPY mobility matvec, N=65536 blobs, a=0.5, xy~U[0,400]^2, z~U[a,3a], f~N(0,1)"
METRIC = "blob-pair interactions/s"
UNIT = "pairs/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "df64"],
                   help="precision of the timed matvec (fp32 is the benchmark line; fp64 and "
                        "df64 for profiling the other kernels)")
    p.add_argument("--clocks-csv", default="",
                   help="keep the nvidia-smi samples of the timed region in this file "
                        "('{rank}' is replaced by the rank; default: a temporary file)")
    p.add_argument("--no-cpu-baseline", action="store_true",
                   help="skip the oracle leg (and with it the accuracy figures)")
    p.add_argument("--no-solve", action="store_true", help="skip the small-suspension solves")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the FP64/df64 matvecs and the monolayer, batch and serving "
                        "sections of the default line")
    p.add_argument("--solves", type=int, default=30)
    p.add_argument("--solve-prec", default="mixed", choices=["mixed", "fp32", "fp64", "df64"],
                   help="precision of the --workload small solves")
    p.add_argument("--precond", default="wall", choices=["wall", "free_shared"],
                   help="block preconditioner of the --workload small / monolayer solves")
    p.add_argument("--workload", choices=["matvec", "small", "monolayer", "batch", "serve",
                                          "resistance", "active", "eval", "setup"],
                   default="matvec",
                   help="matvec: the benchmark line; monolayer / batch / serve: the 663,552-blob "
                        "monolayer solve, 256 batched suspensions and the serving stream, each "
                        "printing its own JSON line; setup: the monolayer's preconditioner "
                        "setup alone")
    p.add_argument("--rate", type=float, default=200.0, help="serving: saturated offered rate")
    p.add_argument("--serve-sat-seconds", type=float, default=0.0,
                   help="serving: arrival window of the saturated run (default 20 s in the "
                        "default line, 60 s for --workload serve)")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="serving: arrival window of each sub-saturation run")
    p.add_argument("--serve-fracs", default="",
                   help="serving: sub-saturation rates as fractions of the measured capacity "
                        "(default 0.8 in the default line, 0.5,0.8 for --workload serve)")
    p.add_argument("--rates", default="",
                   help="serving: fixed offered rates (req/s) instead of --serve-fracs")
    p.add_argument("--tick-pairs", type=float, default=0.0,
                   help="serving: pair evaluations a request may take per tick in the FP32 "
                        "Arnoldi matvec (0 = engine default, < 0 = no limit)")
    p.add_argument("--bodies", type=int, default=4096,
                   help="setup: monolayer bodies (at the monolayer's area density)")
    p.add_argument("--pair-variant", type=int, default=-1,
                   help="FP32 pair-kernel variant (-1 autotune; 0..4 pin one, e.g. for profiling)")
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def max_over_ranks(dist, x: float, device="cpu") -> float:
    """The largest of every rank's x (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(dist, units_local: float, seconds_local: float, device="cpu"):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time.  Returns (rate, max seconds)."""
    t_max = max_over_ranks(dist, seconds_local, device)
    units = float(units_local)
    if dist is not None:
        import torch

        u = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        units = float(u.item())
    return units / t_max, t_max


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous share of n_items independent problems for one rank (the
    first n_items % world ranks take one more)."""
    q, rem = divmod(n_items, world)
    lo = rank * q + min(rank, rem)
    return range(lo, lo + q + (1 if rank < rem else 0))


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(),
                                         f"mb_bench_clocks_{os.getpid()}_gpu{gpu_index}.csv")

    def start(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
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
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, v in enumerate(flags)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def kernel_record(name="pair_kernel_traffic.json"):
    """Counters of one kernel from a committed ncu summary (DRAM bytes per
    launch, FMA-pipe activity), only if the kernel's sources are unchanged
    since the capture (their SHA-256 is recorded beside the numbers)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    for f in rec.get("sources", []):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != rec.get("sha256"):
        return None
    return rec


# ------------------------------------------------------------------ oracle arm
def oracle_pairs_per_s(r, f, a, seconds: float, seed: int = 0):
    """Time the FP64 oracle's double loop on a growing target sample until
    about `seconds` of CPU work; returns (pairs/s, threads, targets, s)."""
    import numpy as np

    from oracle import oracle as O

    n = r.shape[0]
    rng = np.random.default_rng(seed)
    nt = 32
    while True:
        rows = rng.choice(n, min(nt, n), replace=False)
        t0 = time.perf_counter()
        O.matvec(r, f, a, 1.0, True, targets=rows)
        dt = time.perf_counter() - t0
        if dt >= 0.8 * seconds or nt >= n:
            return len(rows) * n / dt, O.num_threads(), len(rows), dt
        nt = int(min(n, max(2 * nt, nt * seconds / max(dt, 1e-3))))


def oracle_rows(r, f, a, n_rows=ORACLE_ROWS, seed=7):
    """The FP64 oracle's product on a seeded subsample of targets (all
    sources), timed: (rows, u_ref rows, seconds, threads)."""
    import numpy as np

    from oracle import oracle as O

    rows = np.sort(np.random.default_rng(seed).choice(r.shape[0], min(n_rows, r.shape[0]),
                                                       replace=False))
    t0 = time.perf_counter()
    ref = O.matvec(r, f, a, 1.0, True, targets=rows)
    return rows, ref, time.perf_counter() - t0, O.num_threads()


def compare_rows(u_rows, ref):
    """Relative L2, max abs and max abs / max |ref| of u against the oracle."""
    import numpy as np

    d = u_rows - ref
    return {"rows": int(ref.shape[0]),
            "rel_l2_vs_oracle": float(np.linalg.norm(d) / np.linalg.norm(ref)),
            "max_abs_vs_oracle": float(np.abs(d).max()),
            "max_abs_over_max_ref": float(np.abs(d).max() / np.abs(ref).max())}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1602_02170_gb300 import inputs as I

    O.build()
    r, f, a = I.config_matvec_cloud(1, n=args.n)
    per_step = max(1.0, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    _, _, nt, _ = oracle_pairs_per_s(r, f, a, per_step)
    import numpy as np

    rng = np.random.default_rng(11)
    for _ in range(args.warmup):
        O.matvec(r, f, a, 1.0, True, targets=rng.choice(args.n, nt, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.matvec(r, f, a, 1.0, True, targets=rng.choice(args.n, nt, replace=False))
    dt = time.perf_counter() - t0
    value = nt * args.n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_blobs": args.n, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{nt} random targets x {args.n} sources per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def measured_peaks(ctx, device):
    """FP32 and FP64 FMA rates measured on this GPU now (TFLOP/s), and its
    SM count read from the device."""
    import torch

    sms = torch.cuda.get_device_properties(device).multi_processor_count
    return {"fp32_tflops": ctx.measure_fma_rate("fp32") / 1e12,
            "fp64_tflops": ctx.measure_fma_rate("fp64") / 1e12, "sm_count": sms,
            "how": "mb_measure_fma_rate: independent FMA chains (f32x2 for FP32) on every SM, "
                   "best of 3 launches, CUDA events, this run"}


def timed_matvec(ctx, r, f, a, prec, steps, warmup, out):
    """Kernel time (ms, from the library's events on the launching stream)
    and step time (ms, CUDA events around each call) of `steps` matvecs."""
    import torch

    for _ in range(warmup):
        ctx.mobility_matvec(r, f, a, 1.0, True, prec, out=out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for e0, e1 in ev:
        e0.record(stream)
        ctx.mobility_matvec(r, f, a, 1.0, True, prec, out=out)
        e1.record(stream)
    torch.cuda.synchronize()
    kms, launches, _ = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    return kms / max(1, launches), sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)

    from paper_1602_02170_gb300 import build as B

    B.build()
    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import inputs as I

    ctx = mb.Context(local)
    if args.pair_variant >= 0:
        ctx.set_pair_variant(args.pair_variant)
    r_np, f_np, a = I.config_matvec_cloud(1 + rank, n=args.n)
    n = args.n
    r = torch.from_numpy(r_np).to(device)
    f = torch.from_numpy(f_np).to(device)
    u = torch.empty_like(r)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)  # 256 MB > L2
    stream = torch.cuda.current_stream(device)
    peaks = measured_peaks(ctx, device)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        ctx.mobility_matvec(r, f, a, 1.0, True, args.prec, out=u)
    torch.cuda.synchronize()
    variant = ctx.pair_variant(n, True) if args.prec == "fp32" else None

    sampler = ClockSampler(local, args.clocks_csv.replace("{rank}", str(rank))
                           if args.clocks_csv else None)
    sampler.start()
    time.sleep(0.3)
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    _, _, launches0 = ctx.profile_read(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        ctx.mobility_matvec(r, f, a, 1.0, True, args.prec, out=u)
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    pair_ms, pair_launches, launches1 = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    t_local = step_ms / 1e3
    pairs_local = float(n) * float(n) * args.steps
    value, t_max = whole_job_rate(dist, pairs_local, t_local, device)
    kernel_avg_s = pair_ms / 1e3 / max(1, pair_launches)
    achieved = FLOPS_PER_PAIR * float(n) * n / kernel_avg_s / 1e12
    u_fp32 = u.cpu().numpy()

    # ---- e2e: host buffers through the C ABI, copies inside the timed region
    r_h = torch.from_numpy(r_np).pin_memory()
    f_h = torch.from_numpy(f_np).pin_memory()
    u_h = torch.empty_like(r_h).pin_memory()
    for _ in range(2):
        ctx.mobility_matvec(r_h, f_h, a, 1.0, True, args.prec, out=u_h)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.mobility_matvec(r_h, f_h, a, 1.0, True, args.prec, out=u_h)
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = whole_job_rate(dist, pairs_local, e2e_s, device)

    nominal = peaks["sm_count"] * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    rec = kernel_record() if args.prec == "fp32" and variant == 3 else None
    if args.prec == "fp32":
        roofline = {
            "bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
            "frac": achieved / peaks["fp32_tflops"],
            "traffic": rec.get("bytes_per_launch_full_size") if rec else None,
            "kernel": KERNEL_NAMES.get(variant, "pair_f32_kernel<wall>"),
            "kernel_ms_avg": 1e3 * kernel_avg_s, "flops_per_pair": FLOPS_PER_PAIR,
            "flops_basis": FLOPS_BASIS,
            "peak_basis": "FP32 FMA rate measured in this run (" + peaks["how"] + "), "
                          f"{peaks['sm_count']} SMs read from the device",
            "peak_nominal": nominal, "frac_of_nominal": achieved / nominal,
            "fma_pipe_active_frac": rec.get("fma_pipe_cycles_active") if rec else None,
            "fma_pipe_basis": "sm__pipe_fma_cycles_active of the committed ncu capture of this "
                              "kernel source (null if the source changed since)"}
    else:
        roofline = {
            "bound": "alu", "achieved": achieved, "peak": peaks["fp64_tflops"],
            "unit": "TFLOP/s (FP64-equivalent)", "frac": achieved / peaks["fp64_tflops"],
            "traffic": None, "kernel_ms_avg": 1e3 * kernel_avg_s,
            "flops_per_pair": FLOPS_PER_PAIR, "flops_basis": FLOPS_BASIS,
            "peak_basis": "FP64 FMA rate measured in this run"}

    # ---- accuracy and the oracle's own rate on the workload's 4,096 targets
    cpu = matvec_err = matvec_fp64 = matvec_df64 = None
    ok = True
    if rank == 0 and not args.no_cpu_baseline:
        rows, ref, dt, threads = oracle_rows(r_np, f_np, a)
        cpu = {"value": len(rows) * n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{len(rows)} random targets x {n} sources ({len(rows) * n:.3g} pairs, "
                         f"{dt:.1f} s)"}
        matvec_err = compare_rows(u_fp32[rows], ref)
        matvec_err.update({"precision": args.prec, "bound_rel_l2": MATVEC_TOL})
        ok = matvec_err["rel_l2_vs_oracle"] <= MATVEC_TOL if args.prec == "fp32" else True
        matvec_err["ok"] = bool(ok)
        if not args.no_extras and args.prec == "fp32":
            out = torch.empty_like(r)
            for prec, steps in (("fp64", 3), ("df64", 5)):
                kms, sms = timed_matvec(ctx, r, f, a, prec, steps, 1, out)
                ach = FLOPS_PER_PAIR * float(n) * n / (kms / 1e3) / 1e12
                line = {"pairs_per_s": float(n) * n / (sms / 1e3), "ms_per_matvec": sms,
                        "kernel_ms_avg": kms, **compare_rows(out.cpu().numpy()[rows], ref),
                        "roofline": {
                            "bound": "alu", "achieved": ach, "peak": peaks["fp64_tflops"],
                            "unit": "TFLOP/s (FP64-equivalent)",
                            "frac": ach / peaks["fp64_tflops"],
                            "flops_per_pair": FLOPS_PER_PAIR,
                            "peak_basis": "FP64 FMA rate measured in this run"}}
                if prec == "fp64":
                    line["kernel"] = "pair_f64sym_kernel<wall> (FP64 pipe, each unordered pair once)"
                    matvec_fp64 = line
                else:
                    line["kernel"] = ("pair_df_kernel<wall> (symmetric, double-float arithmetic "
                                      "on the FP32 pipe)")
                    line["roofline"]["note"] = (
                        "the double-float product runs on the FP32 pipe; frac is its "
                        "FP64-equivalent rate over the FP64 pipe's measured peak, so above 1 "
                        "it outruns any native FP64 kernel")
                    line["roofline"]["fp32_peak"] = peaks["fp32_tflops"]
                    drec = kernel_record("pair_df_kernel_traffic.json")
                    line["roofline"]["fma_pipe_active_frac"] = (
                        drec.get("fma_pipe_cycles_active") if drec else None)
                    matvec_df64 = line

    # ---- mobility solves of the small suspension (latency distribution)
    solve = solve_fp64 = None
    if not args.no_solve and rank == 0:
        solve = bench_solves(ctx, args.solves)
        solve_fp64 = bench_solves(ctx, args.solves, "fp64")

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["monolayer"] = monolayer_line(ctx, "wall", peaks)
        extras["batch"] = batch_line(ctx)
        extras["serve"] = serve_line(ctx, args, sat_seconds=args.serve_sat_seconds or 20.0,
                                     fracs=args.serve_fracs or "0.8")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "df64": "df64"}[args.prec], "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("N=65536", f"N={n}"), "n_blobs": n,
                       "precision":
                       {"fp32": "fp32 pair kernel, hi/lo positions, Kahan-compensated sums, fp64 "
                                "output",
                        "fp64": "fp64 pair kernel",
                        "df64": "double-float symmetric pair kernel"}[args.prec],
                       "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 24 * n,
                    "d2h_bytes_per_step": 24 * n},
            "gpu_launches": int(launches1 - launches0),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "matvec_err": matvec_err,
            "matvec_fp64": matvec_fp64,
            "matvec_df64": matvec_df64,
            "peaks_measured": peaks,
            "solve": solve,
            "solve_fp64": solve_fp64,
            **extras,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0 if ok else 1


def bench_solves(ctx, count, prec="mixed", precond="wall"):
    """Mobility solves of the 8 x 42-blob suspension (tol 1e-10; 1e-6 for fp32)."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_1602_02170_gb300 import inputs as I

    s = I.config_small_suspension(1)
    d = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dt)
    args = (d(s.q), d(s.theta), d(s.blob_start, torch.int64), d(s.rho), d(s.F), d(s.T), s.a,
            s.eta, True)
    tol = 1e-6 if prec == "fp32" else 1e-10
    for _ in range(3):
        ctx.solve_mobility(*args, tol=tol, prec=prec, precond=precond)
    lat = []
    infos = []
    for _ in range(count):
        t0 = time.perf_counter()
        U, W, lam, info = ctx.solve_mobility(*args, tol=tol, prec=prec, precond=precond)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
        infos.append(info)
    # the oracle's dense direct solve of the same problem (blob positions,
    # saddle-point matrix, Cholesky and Schur): the reference values, timed
    t_or = time.perf_counter()
    n_or = 0
    while True:
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, s.eta, True)
        n_or += 1
        if n_or >= 3 or time.perf_counter() - t_or > 2.0:
            break
    t_or = (time.perf_counter() - t_or) / n_or
    eU = float(np.linalg.norm(U.cpu().numpy() - Ur) / np.linalg.norm(Ur))
    eW = float(np.linalg.norm(W.cpu().numpy() - Wr) / np.linalg.norm(Wr))
    lat_ms = sorted(1e3 * x for x in lat)
    return {"workload": f"8 x 42-blob shells above the wall (N=336), GMRES tol {tol:g}, {prec}, "
                        f"{precond} preconditioner",
            "solves_per_s": count / sum(lat), "p50_ms": lat_ms[len(lat_ms) // 2],
            "p99_ms": lat_ms[min(len(lat_ms) - 1, int(math.ceil(0.99 * len(lat_ms))) - 1)],
            "iters": infos[-1]["iters"], "restarts": infos[-1]["restarts"],
            "setup_ms": infos[-1]["setup_ms"], "solve_ms": infos[-1]["solve_ms"],
            "rel_err_U": eU, "rel_err_Omega": eW,
            "oracle_direct_solve": {"solves_per_s": 1.0 / t_or, "kind": "oracle",
                                    "what": "dense FP64 direct solve (numpy/LAPACK), host cores"}}


def bench_small(args):
    """The 8 x 42-blob suspension alone: solves/s, p50/p99 and the setup /
    iteration split of one solve (the command the small-solve launch list
    in profiles/ is taken from)."""
    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B

    B.build()
    ctx = mb.Context(0)
    line = bench_solves(ctx, args.solves, args.solve_prec, args.precond)
    line.update({"metric": "mobility solves/s", "unit": "solves/s", "n_gpus": 1})
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _dev_problem(s):
    import numpy as np
    import torch

    d = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dt)
    return dict(q=d(s.q), theta=d(s.theta), blob_start=d(s.blob_start, torch.int64), rho=d(s.rho),
                F=d(s.F), T=d(s.T))


def precond_factored(blob_counts, sm_count):
    """Whether mb_precond_setup keeps the blocks in factored form: at least
    as many bodies as SMs and blocks of more than 160 rows (up to 2,048)."""
    n = 3 * max(blob_counts)
    return len(blob_counts) >= sm_count and 160 < n <= 2048


def setup_flops(blob_counts, factored=False):
    """FP64 flops of the preconditioner setup (Section 2.2.2), counted per
    body of n = 3 n_p rows as the algorithm is written: the Cholesky factor
    M_p = L L^T (n^3 / 3), and for the explicit inverse also W = L^-1
    (n^3 / 3) and M_p^-1 = W^T W (n^3 / 3)."""
    chol = sum((3.0 * c) ** 3 / 3.0 for c in blob_counts)
    return {"cholesky": chol, "total": chol if factored else 3.0 * chol,
            "form": "factored (L, L^-1 K, N)" if factored else "explicit inverse"}


def monolayer_line(ctx, precond="wall", peaks=None):
    """4,096 shells of 162 blobs (N = 663,552) above the wall, mixed precision
    (FP32 pair kernel in the Krylov iteration, double-float restart
    residuals) to a true relative residual of 1e-8."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_1602_02170_gb300 import inputs as I

    s = I.config_monolayer(1)
    P = _dev_problem(s)
    # size-class autotuning of the FP32 kernel happens on this first matvec
    r = ctx.blob_positions(P["q"], P["theta"], P["blob_start"], P["rho"])
    ctx.mobility_matvec(r, torch.ones_like(r), s.a, 1.0, True, "fp32")
    # the preconditioner setup alone (FP64), timed on the device
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    if precond == "wall":
        ctx.precond_setup(r, P["q"], P["blob_start"], s.a, 1.0, True)
    e1.record()
    torch.cuda.synchronize()
    setup_ms = e0.elapsed_time(e1) if precond == "wall" else None
    t0 = time.perf_counter()
    U, W, lam, info = ctx.solve_mobility(P["q"], P["theta"], P["blob_start"], P["rho"], P["F"],
                                         P["T"], s.a, 1.0, True, tol=1e-8, maxit=300, restart=60,
                                         prec="mixed", precond=precond)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # fresh residual of the returned solution with one double-float product (untimed)
    Ml = ctx.mobility_matvec(r, lam, s.a, 1.0, True, "df64")
    UO = torch.cat([U, W], 1).contiguous()
    rb = ctx.K_apply(r, P["q"], P["blob_start"], UO) - Ml
    rB = ctx.KT_apply(r, P["q"], P["blob_start"], lam) - torch.cat([P["F"], P["T"]], 1)
    fresh = float(torch.sqrt((rb * rb).sum() + (rB * rB).sum()).item())
    rows = np.random.default_rng(3).choice(s.n_blobs, 128, replace=False)
    rr = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    res = O.residual_rows(rows, rr, s.q, s.blob_start, lam.cpu().numpy(), U.cpu().numpy(),
                          W.cpu().numpy(), s.a)
    bnorm = float(np.linalg.norm(np.concatenate([s.F, s.T])))
    line = {"metric": "mobility solves/s", "workload": "monolayer: 4096 x 162-blob shells, "
            "N=663552, a=0.12, 200x200 patch, z in [1.2,1.6]", "value": 1.0 / dt,
            "unit": "solves/s", "seconds": dt, "tol": 1e-8, "prec": "mixed (fp32 + df64 residual)",
            "precond": precond, "precond_bytes": ctx.workspace_bytes(),
            "info": info, "pairs_per_matvec": float(s.n_blobs) ** 2,
            "fresh_df64_rel_residual": fresh / bnorm,
            "oracle_sampled_residual_rows_max_over_bnorm": float(np.abs(res).max() / bnorm),
            "oracle_rows": int(len(rows)), "n_gpus": 1}
    if setup_ms is not None:
        counts = np.diff(s.blob_start)
        fl = setup_flops(counts, precond_factored(counts, peaks["sm_count"] if peaks else 152))
        st = {"ms": setup_ms, "fp64_flops": fl["total"], "cholesky_flops": fl["cholesky"],
              "form": fl["form"], "achieved_tflops": fl["total"] / (setup_ms / 1e3) / 1e12,
              "what": "mb_precond_setup alone: assembly, Cholesky with L^-1 K, the Schur "
                      "complement (and for the explicit form L^-1 and M^-1) of every body, "
                      "CUDA events"}
        if peaks:
            st["fp64_peak_tflops"] = peaks["fp64_tflops"]
            st["frac"] = st["achieved_tflops"] / peaks["fp64_tflops"]
        line["precond_setup"] = st
    return line


def bench_monolayer(args):
    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B

    B.build()
    ctx = mb.Context(0)
    peaks = measured_peaks(ctx, 0)
    print(json.dumps(monolayer_line(ctx, args.precond, peaks)), flush=True)
    ctx.close()
    return 0


def bench_setup(args):
    """The monolayer's preconditioner setup alone, three times, then ten
    applications of it (the command the setup and apply kernels' launch list
    and captures are taken from); --bodies shrinks the patch at the same
    density."""
    import numpy as np
    import torch

    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B
    from paper_1602_02170_gb300 import inputs as I

    B.build()
    ctx = mb.Context(0)
    peaks = measured_peaks(ctx, 0)
    s = I.config_monolayer(1, n_bodies=args.bodies,
                           box=200.0 * math.sqrt(args.bodies / 4096.0))
    P = _dev_problem(s)
    r = ctx.blob_positions(P["q"], P["theta"], P["blob_start"], P["rho"])
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.precond_setup(r, P["q"], P["blob_start"], s.a, 1.0, True)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    counts = np.diff(s.blob_start)
    fl = setup_flops(counts, precond_factored(counts, peaks["sm_count"]))
    ms = min(times)
    rng = np.random.default_rng(0)
    w = torch.as_tensor(rng.standard_normal((s.n_blobs, 3))).cuda()
    g = torch.as_tensor(rng.standard_normal((s.n_bodies, 6))).cuda()
    ctx.precond_apply(w, g)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        ctx.precond_apply(w, g)
    e1.record()
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / 10
    nrows = 3.0 * counts
    apply_fma = float(np.sum((nrows + 6.0) ** 2))
    print(json.dumps({"metric": "preconditioner setup ms", "workload": f"monolayer blocks, "
                      f"{s.n_bodies} x 486 rows, wall", "ms": times, "form": fl["form"],
                      "fp64_flops": fl["total"],
                      "achieved_tflops": fl["total"] / (ms / 1e3) / 1e12,
                      "fp64_peak_tflops": peaks["fp64_tflops"],
                      "frac": fl["total"] / (ms / 1e3) / 1e12 / peaks["fp64_tflops"],
                      "apply_ms": apply_ms,
                      "apply_tflops": 2.0 * apply_fma / (apply_ms / 1e3) / 1e12,
                      "apply_frac": 2.0 * apply_fma / (apply_ms / 1e3) / 1e12 / peaks["fp64_tflops"],
                      "apply_flops_basis": "(n + 6)^2 FP64 FMA per body and application",
                      "n_gpus": 1}), flush=True)
    ctx.close()
    return 0


def bench_resistance(args):
    """Iterations and time of the resistance problem (Eq. resistance_problem)
    beside the mobility problem, for growing suspensions of 42-blob shells in
    an unbounded domain at volume fraction 0.1 (mixed precision, tol 1e-8).
    Section 4.4 reports resistance iterations growing like N^(1/3) while the
    mobility problem's stay flat; the fitted exponent is printed."""
    import numpy as np
    import torch

    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B
    from paper_1602_02170_gb300 import inputs as I

    B.build()
    ctx = mb.Context(0)
    a, R, phi = 0.243, 1.0, 0.1
    rows = []
    for nb in (8, 64, 512, 2048):
        box = (nb * 4.0 / 3.0 * math.pi * (R + a) ** 3 / phi) ** (1.0 / 3.0)
        s = I.sphere_suspension(17 + nb, nb, 42, a, box, R + a + 0.05, R + a + 0.05 + box)
        P = _dev_problem(s)
        rng = np.random.default_rng(nb)
        U = torch.as_tensor(rng.standard_normal((nb, 3))).cuda()
        W = torch.as_tensor(0.5 * rng.standard_normal((nb, 3))).cuda()
        row = {"n_bodies": nb, "n_blobs": int(s.n_blobs)}
        for kind in ("mobility", "resistance"):
            def run():
                if kind == "mobility":
                    return ctx.solve_mobility(P["q"], P["theta"], P["blob_start"], P["rho"],
                                              P["F"], P["T"], a, 1.0, False, tol=1e-8,
                                              maxit=2000, restart=100, prec="mixed")
                return ctx.solve_resistance(P["q"], P["theta"], P["blob_start"], P["rho"], U, W, a,
                                            1.0, False, tol=1e-8, maxit=2000, restart=100,
                                            prec="mixed")
            run()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = run()
            torch.cuda.synchronize()
            row[kind] = {"iters": out[3]["iters"], "restarts": out[3]["restarts"],
                         "seconds": time.perf_counter() - t0,
                         "rel_residual": out[3]["rel_residual"]}
        rows.append(row)
    n = np.array([r["n_blobs"] for r in rows], dtype=float)
    fit = {k: float(np.polyfit(np.log(n), np.log([r[k]["iters"] for r in rows]), 1)[0])
           for k in ("mobility", "resistance")}
    line = {"metric": "GMRES iterations vs N, resistance and mobility problems",
            "workload": "42-blob shells (a=0.243) in an unbounded domain, volume fraction 0.1, "
                        "mixed precision, tol 1e-8, restart 100",
            "rows": rows, "fitted_exponent_iters_vs_N": fit, "n_gpus": 1}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def bench_active(args):
    """Active slip on single shells in an unbounded domain: the squirmer's
    speed against (2/3) B1 (Section 4.3) and the stresslet radius R_s under
    the strain slip (Section 4.1), with solve times (FP64, tol 1e-10)."""
    import numpy as np
    import torch

    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B
    from paper_1602_02170_gb300 import inputs as I

    B.build()
    ctx = mb.Context(0)
    d = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dt)
    rows = []
    for n in (42, 162, 642):
        rho = I.shell(n)
        a = 0.5 * I.min_spacing(rho)
        th = np.arccos(np.clip(rho[:, 2] / np.linalg.norm(rho, axis=1), -1.0, 1.0))
        ph = np.arctan2(rho[:, 1], rho[:, 0])
        e_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
        squirm = np.sin(th)[:, None] * e_th
        strain = -np.stack([rho[:, 0], -rho[:, 1], np.zeros(n)], axis=1)
        body = (d(np.zeros((1, 3))), d([[1.0, 0, 0, 0]]), d([0, n], torch.int64), d(rho))
        z = d(np.zeros((1, 3)))
        row = {"n_blobs": n, "a_over_Rg": a}
        for name, slip in (("squirmer", squirm), ("strain", strain)):
            ctx.solve_mobility(*body, z, z, a, 1.0, False, d(slip), tol=1e-10, prec="fp64")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            U, W, lam, info = ctx.solve_mobility(*body, z, z, a, 1.0, False, d(slip), tol=1e-10,
                                                 prec="fp64")
            torch.cuda.synchronize()
            row[name + "_ms"] = 1e3 * (time.perf_counter() - t0)
            if name == "squirmer":
                uz = float(U[0, 2])
                row["squirmer_speed_over_2B1_3"] = uz / (2.0 / 3.0)
                row["squirmer_rel_err_over_a"] = (uz / (2.0 / 3.0) - 1.0) / a
            else:
                S = ctx.lambda_moments(body[3], body[0], body[2], lam)[0].cpu().numpy()
                s = 0.5 * (S + S.T) - np.trace(S) / 3.0 * np.eye(3)
                row["Rs_over_Rg"] = float((-3.0 * s[0, 0] / (20.0 * math.pi)) ** (1.0 / 3.0))
        rows.append(row)
    print(json.dumps({"metric": "active slip: squirmer speed and stresslet radius",
                      "workload": "single icosahedral shells, a = s/2, unbounded domain, FP64, "
                                  "tol 1e-10", "rows": rows, "n_gpus": 1}), flush=True)
    ctx.close()
    return 0


def bench_eval(args):
    """Flow evaluation away from the blobs: 65,536 tracer points over the
    65,536-blob matvec cloud (FP32 packed kernel), and the Appendix B
    rendering of the same points with every blob split into 12."""
    import torch

    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B
    from paper_1602_02170_gb300 import inputs as I

    B.build()
    ctx = mb.Context(0)
    r_np, f_np, a = I.config_matvec_cloud(1, 65536)
    x_np, _, _ = I.config_matvec_cloud(2, 65536)
    r, f, x = (torch.from_numpy(v).cuda() for v in (r_np, f_np, x_np))
    off = torch.from_numpy(I.shell(12) * a).cuda()
    out = {}
    for name, call, pairs in (
            ("eval", lambda: ctx.mobility_eval(x, r, f, a, 1.0, True, "fp32"), 65536.0 ** 2),
            ("render_12", lambda: ctx.render_flow(x, r, f, off, 0.25 * a, 1.0, True, "fp32"),
             65536.0 * 65536.0 * 12)):
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            call()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / 5
        out[name] = {"ms": 1e3 * dt, "pairs_per_s": pairs / dt}
    print(json.dumps({"metric": "flow evaluation pairs/s", "workload": "65,536 points x 65,536 "
                      "blobs (C2 cloud), wall, FP32; rendering with 12 sub-blobs per blob",
                      **out, "n_gpus": 1}), flush=True)
    ctx.close()
    return 0


def batch_line(ctx, dist=None, rank=0, world=1, local=0):
    """256 independent mixed suspensions (42-blob shells and 15-blob
    boomerangs, log-uniform 8..2048 bodies) solved together, mixed precision
    to 1e-8; compared on a random subset with the plain FP64 path solving one
    problem at a time, at the same tolerance.  Under torchrun the problems
    are split into contiguous shares, one per rank (no collective on the data
    path); the rate is all problems over the slowest rank's time.  Returns
    the line on rank 0 (None elsewhere)."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_1602_02170_gb300 import inputs as I

    t0 = time.perf_counter()
    susp = I.config_batched(1)
    gen_s = time.perf_counter() - t0
    mine = list(shard(len(susp), rank, world))
    probs = {k: _dev_problem(susp[k]) for k in mine}
    a = susp[0].a
    ctx.solve_batch([probs[k] for k in mine[:4]], a, tol=1e-8, prec="mixed")  # warm-up
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    res_list = ctx.solve_batch([probs[k] for k in mine], a, tol=1e-8, maxit=300, restart=60,
                               prec="mixed")
    torch.cuda.synchronize()
    t_local = time.perf_counter() - t0
    rate, t_batch = whole_job_rate(dist, len(mine), t_local, torch.device("cuda", local))
    res = dict(zip(mine, res_list))
    iters = [r[3]["iters"] for r in res_list]
    if rank != 0:
        return None
    rng = np.random.default_rng(5)
    sub = sorted(rng.choice(mine, min(8, len(mine)), replace=False).tolist())
    t0 = time.perf_counter()
    sub_batch = ctx.solve_batch([probs[k] for k in sub], a, tol=1e-8, prec="mixed")
    torch.cuda.synchronize()
    t_sub_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    sub_fp64 = []
    for k in sub:
        P = probs[k]
        sub_fp64.append(ctx.solve_mobility(P["q"], P["theta"], P["blob_start"], P["rho"], P["F"],
                                           P["T"], a, 1.0, True, tol=1e-8, maxit=300, restart=60,
                                           prec="fp64"))
    torch.cuda.synchronize()
    t_sub_fp64 = time.perf_counter() - t0
    rel = lambda x, y: float(((x - y).norm() / y.norm()).item())
    diff_full = max(rel(res[k][0], y[0]) for k, y in zip(sub, sub_fp64))
    diff_sub = max(rel(x[0], y[0]) for x, y in zip(sub_batch, sub_fp64))
    oracle_err = []
    for k in sub:
        s = susp[k]
        if s.n_blobs <= 1500:
            rr = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
            Ur, _, _ = O.solve_saddle(rr, s.q, s.blob_start, s.F, s.T, a, 1.0, True)
            oracle_err.append(float(np.linalg.norm(res[k][0].cpu().numpy() - Ur) / np.linalg.norm(Ur)))
    pairs = float(sum(s.n_blobs ** 2 for s in susp))
    return {"metric": "mobility solves/s", "workload": "batched: 256 mixed suspensions "
            "(42-blob shells / 15-blob boomerangs, a=0.1625), bodies log-uniform 8..2048, "
            "z in [1.2,3]", "value": rate, "unit": "solves/s", "seconds": t_batch,
            "tol": 1e-8, "prec": "mixed (fp32 + df64 residual), one batched launch per kernel",
            "n_blobs_total": int(sum(s.n_blobs for s in susp)),
            "n_bodies_total": int(sum(s.n_bodies for s in susp)),
            "pairs_per_batched_matvec": pairs, "iters_median_rank0": float(np.median(iters)),
            "iters_max_rank0": int(max(iters)), "converged_all": all(
                r[3]["converged"] == 1 for r in res_list), "generation_s": gen_s,
            "subset": {"problems": sub, "batched_mixed_solves_per_s": len(sub) / t_sub_batch,
                       "fp64_one_at_a_time_solves_per_s": len(sub) / t_sub_fp64,
                       "max_rel_diff_U_full_batch_vs_fp64": diff_full,
                       "max_rel_diff_U_subset_batch_vs_fp64": diff_sub,
                       "oracle_rel_err_U_small_problems": oracle_err},
            "n_gpus": world, "scaling": "strong",
            "parallelism": "problems split across ranks" if world > 1 else "single GPU"}


def bench_batch(args):
    import torch

    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B

    rank, world, local = dist_info()
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    B.build()
    ctx = mb.Context(local)
    line = batch_line(ctx, dist, rank, world, local)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
    ctx.close()
    return 0


def _gen_requests(seeds):
    """Serving requests (one seeded mixed suspension each), generated on the
    host cores by a pool of spawned processes."""
    import multiprocessing as mp

    from paper_1602_02170_gb300 import inputs as I

    seeds = [int(x) for x in seeds]
    workers = max(1, min(16, (os.cpu_count() or 2) - 2))
    if len(seeds) < 16 or workers == 1:
        return [I.config_serving_request(x) for x in seeds]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(I.config_serving_request, seeds, chunksize=8)


def _serve_run(ctx, a, probs, arrivals, window, drain, tick_pairs, keep_results=False):
    """Serve `probs` arriving at `arrivals` (seconds) on a fresh server; each
    request's data goes to the device when it arrives.  Latency runs from the
    scheduled arrival to the tick that sees the request done."""
    import numpy as np

    import paper_1602_02170_gb300 as mb

    srv = mb.Server(ctx, a, tol=1e-8, prec="mixed", restart=30, max_blobs=4_000_000,
                    max_bodies=150_000, max_precond_bytes=12 << 30, max_requests=512,
                    tick_pairs=tick_pairs)
    inflight, lat, done_blobs, results, work, its = {}, [], [], {}, 0.0, []
    nsub = failed = 0
    queue_at_window = None
    max_outstanding = 0
    start = time.perf_counter()
    ticks = 0
    while True:
        now = time.perf_counter() - start
        while nsub < len(arrivals) and arrivals[nsub] <= now:
            P = _dev_problem(probs[nsub])
            t, outs = srv.submit(P)
            inflight[t] = (arrivals[nsub], nsub, outs)
            nsub += 1
        nr, nq = srv.step()
        ticks += 1
        now = time.perf_counter() - start
        for t in srv.finished():
            st_, info, status = srv.poll(t)
            arr, k, outs = inflight.pop(t)
            if st_ == mb.Server.DONE and status == "MB_OK":
                its.append(info["iters"])
                lat.append(now - arr)
                done_blobs.append(probs[k].n_blobs)
                work += request_work(probs[k].n_blobs, info["iters"])
                if keep_results:
                    results[k] = (outs[0].clone(), outs[1].clone())
            else:
                failed += 1
        max_outstanding = max(max_outstanding, len(inflight))
        if queue_at_window is None and now >= window:
            queue_at_window = len(inflight) + (len(arrivals) - nsub)
        if now >= window and (not drain or (not inflight and nsub == len(arrivals))):
            break
        if nr == 0 and nq == 0 and nsub < len(arrivals):
            time.sleep(max(0.0, min(arrivals[nsub] - now, 0.01)))
    wall = time.perf_counter() - start
    srv.close()
    lat_ms = sorted(1e3 * x for x in lat)
    pct = lambda q: lat_ms[min(len(lat_ms) - 1, int(math.ceil(q * len(lat_ms))) - 1)] if lat_ms else None
    return {"window_s": window, "wall_s": wall, "offered": int(len(arrivals)),
            "offered_per_s": len(arrivals) / window if window > 0 else None, "served": len(lat),
            "served_per_s": len(lat) / wall, "failed": failed, "p50_ms": pct(0.5),
            "p99_ms": pct(0.99), "outstanding_at_window_end": queue_at_window,
            "max_outstanding": max_outstanding, "unserved_at_end": int(len(arrivals) - len(lat)),
            "ticks": ticks, "mean_served_blobs": float(np.mean(done_blobs)) if done_blobs else None,
            "served_work_pairs": work,
            "iters_median": float(np.median(its)) if its else None,
            "mean_offered_blobs": float(np.mean([p.n_blobs for p in probs])) if probs else None,
            "_results": results}


# One mixed-precision request costs, in pair evaluations, N^2 per FP32 Krylov
# iteration plus the double-float product of its first refinement residual,
# which takes about 8 FP32 matvecs on this GPU (58.5 vs 7.45 ms at N = 65,536).
DF64_MATVEC_EQUIV = 8.0


def request_work(n_blobs, iters):
    return float(n_blobs) ** 2 * (iters + DF64_MATVEC_EQUIV)


def serve_line(ctx, args, sat_seconds, fracs):
    """The serving stream (Poisson arrivals, blob counts log-uniform in
    [100, 2e5], mixed shells and boomerangs, one freshly seeded problem per
    request): saturated at args.rate req/s over `sat_seconds`; the capacity
    measured by serving 64 requests submitted at once; then drained runs at
    fractions of that capacity over args.serve_seconds each, with p50/p99
    latency, served vs offered and the queue at the end of the window; and
    sampled requests of the last run solved alone against their served
    result (and the oracle's direct solve for a small one)."""
    import numpy as np
    import torch

    from oracle import oracle as O

    out = {"metric": "mobility solves/s and p99 latency",
           "workload": "serving: Poisson arrivals, blobs log-uniform 100..2e5 (mixed 42-blob "
                       "shells / 15-blob boomerangs, a=0.1625), one seeded problem per request",
           "tol": 1e-8, "prec": "mixed (fp32 + df64 residual)", "tick_pairs": args.tick_pairs,
           "n_gpus": 1}
    # saturated: the offered load of the workload
    rng = np.random.default_rng(1)
    arr = np.cumsum(rng.exponential(1.0 / args.rate, int(args.rate * sat_seconds * 2) + 16))
    arr = arr[arr < sat_seconds]
    t0 = time.perf_counter()
    probs = _gen_requests(10_000_000 + np.arange(len(arr)))
    gen_s = time.perf_counter() - t0
    a = probs[0].a
    sat = _serve_run(ctx, a, probs, arr, sat_seconds, False, args.tick_pairs)
    sat.pop("_results")
    sat["rate_offered"] = args.rate
    sat["generation_s"] = gen_s
    out["saturated"] = sat
    del probs
    # capacity: the engine's rate of pair work with 64 requests submitted at
    # once and served to completion, over the mean work of a request of the
    # offered mix.  Work per request grows like N^2 over a heavy-tailed size
    # distribution, so a request count from a small sample would misjudge it.
    cap_probs = _gen_requests(20_000_000 + np.arange(64))
    cap = _serve_run(ctx, a, cap_probs, np.zeros(64), 0.0, True, args.tick_pairs)
    cap.pop("_results")
    work_rate = cap["served_work_pairs"] / cap["wall_s"]
    mix = _gen_requests(40_000_000 + np.arange(512))
    iters_typ = cap["iters_median"] or 15.0
    mean_work = float(np.mean([request_work(p.n_blobs, iters_typ) for p in mix]))
    capacity = work_rate / mean_work
    del mix
    out["capacity"] = {"solves_per_s": capacity, "pair_work_per_s": work_rate,
                       "mean_work_pairs_per_request": mean_work, "requests": 64,
                       "wall_s": cap["wall_s"], "iters_median": iters_typ,
                       "how": "pair work per second (N^2 per Krylov iteration plus 8 N^2 for the "
                              "double-float residual) of 64 fresh requests submitted at once and "
                              "served to completion, over the mean work of 512 requests drawn "
                              "from the offered distribution"}
    rates = ([float(x) for x in args.rates.split(",")] if args.rates
             else [float(x) * capacity for x in fracs.split(",")])
    subs = []
    for i, rate in enumerate(rates):
        rng = np.random.default_rng(100 + i)
        arr = np.cumsum(rng.exponential(1.0 / rate, int(rate * args.serve_seconds * 2) + 16))
        arr = arr[arr < args.serve_seconds]
        probs = _gen_requests((30 + i) * 1_000_000 + np.arange(len(arr)))
        last = i == len(rates) - 1
        run = _serve_run(ctx, a, probs, arr, args.serve_seconds, True, args.tick_pairs,
                         keep_results=last)
        results = run.pop("_results")
        run["rate_offered"] = rate
        if not args.rates:
            run["fraction_of_capacity"] = rate / capacity
        if last and results:
            # sampled requests alone vs in the mix: smallest, median and largest served
            order = sorted(results, key=lambda k: probs[k].n_blobs)
            picks = sorted({order[0], order[len(order) // 2], order[-1]})
            worst = 0.0
            for k in picks:
                P = _dev_problem(probs[k])
                U = ctx.solve_mobility(P["q"], P["theta"], P["blob_start"], P["rho"], P["F"],
                                       P["T"], a, 1.0, True, tol=1e-8, maxit=300, restart=30,
                                       prec="mixed")[0]
                worst = max(worst, float(((results[k][0] - U).norm() / U.norm()).item()))
            run["alone_vs_served_max_rel_diff_U"] = worst
            run["alone_vs_served_requests"] = [int(probs[k].n_blobs) for k in picks]
            s = probs[order[0]]
            if s.n_blobs <= 1500:
                rr = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
                Ur, _, _ = O.solve_saddle(rr, s.q, s.blob_start, s.F, s.T, a, 1.0, True)
                run["oracle_rel_err_U_smallest"] = float(
                    np.linalg.norm(results[order[0]][0].cpu().numpy() - Ur) / np.linalg.norm(Ur))
        subs.append(run)
        del probs
    torch.cuda.synchronize()
    out["sub_saturation"] = subs
    out["value"] = subs[-1]["served_per_s"] if subs else sat["served_per_s"]
    out["p99_ms"] = subs[-1]["p99_ms"] if subs else sat["p99_ms"]
    out["unit"] = "solves/s"
    return out


def bench_serve(args):
    import paper_1602_02170_gb300 as mb
    from paper_1602_02170_gb300 import build as B

    B.build()
    ctx = mb.Context(0)
    line = serve_line(ctx, args, sat_seconds=args.serve_sat_seconds or 60.0,
                      fracs=args.serve_fracs or "0.5,0.8")
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "small":
        return bench_small(args)
    if args.workload == "resistance":
        return bench_resistance(args)
    if args.workload == "active":
        return bench_active(args)
    if args.workload == "eval":
        return bench_eval(args)
    if args.workload == "monolayer":
        return bench_monolayer(args)
    if args.workload == "batch":
        return bench_batch(args)
    if args.workload == "serve":
        return bench_serve(args)
    if args.workload == "setup":
        return bench_setup(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
