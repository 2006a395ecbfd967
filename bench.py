#!/usr/bin/env python
"""Benchmark of the wall-corrected RPY pair kernel (blob-pair interactions/s).

Workload: the wall-RPY mobility product u = M f for N = 65,536 free blobs,
a = 0.5, x, y ~ U[0, 400], z ~ U[a, 3a], f ~ N(0, 1) (seeded, synthetic).
One step = one mb_mobility_matvec call (FP32 pair kernel with hi/lo
positions and Kahan-compensated accumulation) on inputs already in HBM; the
L2 is flushed (256 MB write) before every timed step.  Pairs per step = N^2
(self pairs included).

Also reported on the same line:
  e2e          the same metric through the C ABI with host buffers (pinned):
               host->device copies of r and f and the device->host copy of u
               inside the timed region of every step
  roofline     the pair kernel against the FP32 ALU peak (152 SMs x 128 FP32
               lanes x 2 flop x 2.07 GHz), algorithmic flops per pair as
               written in the kernel's formula
  cpu_baseline the FP64 oracle on this host's cores, on a bounded sample
  solve        mobility solves of 8 x 42-blob shells (the small suspension),
               solves/s and p50/p99 latency, error vs the oracle

--impl reference times the FP64 oracle (the reference arm of this repo) on
this host's cores on the same workload, a bounded sample of targets per step.
Multi-GPU: `--gpus N` under torchrun runs N independent replicas (the path is
not sharded here); value = pairs of all ranks / slowest rank's time.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 65536
# Arithmetic in the kernel's per-pair formula (rpy_wall.cuh, pair_accumulate
# with the wall, plus the hi/lo separation): multiplies and adds counted
# separately, rsqrt as one; the rare overlap branch is not counted.
FLOPS_PER_PAIR = 117
FP32_LANES_PER_SM = 128
SMS = 152
SM_MAX_MHZ = 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
KERNEL_NAMES = {0: "pair_f32_kernel<wall> (scalar, 1 target/thread)",
                1: "pair_f32x2_kernel<wall,1> (packed f32x2, 2 targets/thread)",
                2: "pair_f32x2_kernel<wall,2> (packed f32x2, 4 targets/thread)"}
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
    p.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-solve", action="store_true")
    p.add_argument("--solves", type=int, default=30)
    return p.parse_args()


# ------------------------------------------------------------------ helpers
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

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
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


def traffic_for_kernel():
    """Per-launch DRAM bytes of the pair kernel from the committed ncu summary,
    only if the kernel source is unchanged since it was captured."""
    path = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    for f in rec.get("sources", []):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != rec.get("sha256"):
        return None
    return rec.get("bytes_per_launch_full_size")


# ------------------------------------------------------------------ oracle arm
def oracle_pairs_per_s(r, f, a, seconds: float, seed: int = 0):
    """Time the FP64 oracle's double loop on a growing target sample until
    about `seconds` of CPU work; returns (pairs/s, threads, targets)."""
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
    r_np, f_np, a = I.config_matvec_cloud(1 + rank, n=args.n)
    n = args.n
    r = torch.from_numpy(r_np).to(device)
    f = torch.from_numpy(f_np).to(device)
    u = torch.empty_like(r)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)  # 256 MB > L2
    stream = torch.cuda.current_stream(device)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        ctx.mobility_matvec(r, f, a, 1.0, True, args.prec, out=u)
    torch.cuda.synchronize()
    variant = ctx.pair_variant(n, True) if args.prec == "fp32" else None

    sampler = ClockSampler(local)
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
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    pairs = float(n) * float(n) * args.steps * world
    value = pairs / t_max
    kernel_avg_s = pair_ms / 1e3 / max(1, pair_launches)
    achieved = FLOPS_PER_PAIR * float(n) * n / kernel_avg_s / 1e12

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
    te = torch.tensor([e2e_s], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = pairs / float(te.item())

    # ---- mobility solves of the small suspension (latency distribution)
    solve = None
    if not args.no_solve and rank == 0:
        solve = bench_solves(ctx, args.solves)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        pps, cores, nt, dt = oracle_pairs_per_s(r_np, f_np, a, args.cpu_seconds)
        cpu = {"value": pps, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nt} random targets x {n} sources ({nt * n:.3g} pairs, {dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_blobs": n, "precision":
                       "fp32 pair kernel, hi/lo positions, Kahan-compensated sums, fp64 output"
                       if args.prec == "fp32" else "fp64 pair kernel",
                       "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                         "traffic": traffic_for_kernel(),
                         "kernel": KERNEL_NAMES.get(variant, "pair_f64_kernel<wall>"),
                         "kernel_ms_avg": 1e3 * kernel_avg_s,
                         "flops_per_pair": FLOPS_PER_PAIR,
                         "peak_basis": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (max SM clock)",
                         "frac_at_measured_clock": (achieved / (FP32_PEAK_TFLOPS * clocks["sm_mhz"]
                                                                / SM_MAX_MHZ))
                         if clocks else None},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 24 * n,
                    "d2h_bytes_per_step": 24 * n},
            "gpu_launches": int(launches1 - launches0),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "solve": solve,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def bench_solves(ctx, count):
    """Mixed-precision mobility solves of the 8 x 42-blob suspension."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_1602_02170_gb300 import inputs as I

    s = I.config_small_suspension(1)
    d = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dt)
    args = (d(s.q), d(s.theta), d(s.blob_start, torch.int64), d(s.rho), d(s.F), d(s.T), s.a,
            s.eta, True)
    for _ in range(3):
        ctx.solve_mobility(*args, tol=1e-10, prec="mixed")
    lat = []
    infos = []
    for _ in range(count):
        t0 = time.perf_counter()
        U, W, lam, info = ctx.solve_mobility(*args, tol=1e-10, prec="mixed")
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
        infos.append(info)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, s.eta, True)
    eU = float(np.linalg.norm(U.cpu().numpy() - Ur) / np.linalg.norm(Ur))
    eW = float(np.linalg.norm(W.cpu().numpy() - Wr) / np.linalg.norm(Wr))
    lat_ms = sorted(1e3 * x for x in lat)
    return {"workload": "8 x 42-blob shells above the wall (N=336), GMRES tol 1e-10, mixed precision",
            "solves_per_s": count / sum(lat), "p50_ms": lat_ms[len(lat_ms) // 2],
            "p99_ms": lat_ms[min(len(lat_ms) - 1, int(math.ceil(0.99 * len(lat_ms))) - 1)],
            "iters": infos[-1]["iters"], "rel_err_U": eU, "rel_err_Omega": eW}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
