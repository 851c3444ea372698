#!/usr/bin/env python3
"""Throughput benchmark of the differentiable cloth hot path on GB300.

Metric: cloth time steps per second, forward + adjoint, FP64.
One bench step = one full rollout of the draped-cloth workload (61 x 61 grid,
3721 nodes, 7200 triangles, dropped over a sphere of radius 0.3 m and the
ground; 125 time steps at h = 1/120 s, 20 PD iterations per step) forward, then
its gradient w.r.t. (x0, v0, k_stretch, k_bend, mu) through the
torch.autograd.Function with checkpoints every 25 steps.  Inputs are synthetic
and seeded (scenes.draped_cloth).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it is launched by torch.distributed.run, one rank per GPU; every rank
runs its own replica of the workload (replicas only: the path has no exchange
step) and rank 0 prints one JSON line.  `--impl reference` times the plain
FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cloth time steps/sec (fwd+adjoint, FP64)"
UNIT = "cloth_steps/s"
N_STEPS = 125
CHECKPOINT_EVERY = 25
L2_FLUSH_BYTES = 512 << 20        # > 129 MB L2
WORKLOAD = ("draped cloth 61x61 (3721 nodes, 7200 triangles), sphere r=0.3 m + ground plane, "
            "125 steps at h=1/120 s, 20 PD iterations/step, forward + checkpointed adjoint (every 25 steps), "
            "gradient w.r.t. x0, v0, k_stretch, k_bend, mu")

# FP32 CUDA-core peak from unit counts and the maximum SM clock (GB300: 152 SMs,
# 128 FP32 lanes per SM, FMA = 2 flops, 2070 MHz); FP64 nominal 1.25 TFLOP/s.
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25

# DRAM traffic per launch of the roofline kernel from the ncu capture summarised in
# profiles/ (null when the kernel source changed since the capture).
TRAFFIC = {"front": {"bytes": None, "source_sha": None}}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--roofline-kernel", default="front")
    ap.add_argument("--rollout-steps", type=int, default=N_STEPS,
                    help="cloth steps per rollout (125 for the workload; ncu launch lists use a shorter rollout)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def aggregate(local_ms: float, world: int):
    """Max of the per-rank timed milliseconds over all ranks (barrier semantics)."""
    if world == 1:
        return local_ms
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle sample

def oracle_sample(n_fwd: int = 5, n_adj: int = 1, start_step: int = 20):
    """Time the CPU oracle on a bounded sample of the workload: n_fwd forward steps
    and n_adj adjoint steps of the 61x61 draped cloth starting at `start_step`
    (reached untimed).  Returns (steps/s for fwd+adjoint, seconds timed, sample text)."""
    import scenes
    from oracle import cloth as oc
    sc = scenes.draped_cloth()
    M = oc.model_from_scene(sc)
    x, v = sc.x0, sc.v0
    for _ in range(start_step):
        x, v, _ = oc.step(M, x, v)
    t0 = time.perf_counter()
    recs = []
    for _ in range(n_fwd):
        x, v, rec = oc.step(M, x, v)
        recs.append(rec)
    t1 = time.perf_counter()
    gx, gv = sc.loss_w, sc.loss_w * 0.0
    for rec in recs[::-1][:n_adj]:
        gx, gv, _, _, _ = oc.adjoint_step(M, rec, gx, gv)
    t2 = time.perf_counter()
    per_step = (t1 - t0) / n_fwd + (t2 - t1) / n_adj
    sample = (f"oracle (numpy/scipy FP64, banded Cholesky + direct sparse KKT adjoint) on the 61x61 draped "
              f"cloth: {n_fwd} forward steps and {n_adj} adjoint step(s) from step {start_step}; "
              f"steps/s = 1 / (forward s/step + adjoint s/step)")
    return 1.0 / per_step, t2 - t0, sample


def cpu_baseline_subprocess():
    """Run the oracle sample single-threaded in a child process."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample"], env=env,
                       capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------- our arm

def kernel_sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def run_ours(args):
    import torch

    import paper_2106_05306_gb300 as dc
    import scenes
    from paper_2106_05306_gb300 import build as dcbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl")
    dcbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sc = scenes.draped_cloth()
    p = sc.params
    cloth = dc.Cloth(sc.rest_pos, sc.tris, sc.pins, device=dev)
    cloth.set_params(k_stretch=p.k_stretch, k_bend=p.k_bend, density=p.density, mu=p.mu, h=p.h, gravity=p.gravity,
                     contact_margin=p.contact_margin, n_pd_iters=p.n_pd_iters, obstacles=sc.obstacles,
                     checkpoint_every=CHECKPOINT_EVERY)
    x0 = torch.tensor(sc.x0, device=dev)
    v0 = torch.tensor(sc.v0, device=dev)
    xi = torch.tensor(sc.loss_w, device=dev)
    theta = torch.tensor([p.k_stretch, p.k_bend, p.mu], dtype=torch.float64, requires_grad=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    n_cloth = args.rollout_steps

    def one_step():
        a = x0.detach().requires_grad_(True)
        b = v0.detach().requires_grad_(True)
        xN, vN = dc.rollout_fn(cloth, a, b, theta, n_cloth)
        L = (xN * xi).sum()
        L.backward()
        return a.grad, b.grad

    for _ in range(max(args.warmup, 0)):
        one_step()
    torch.cuda.synchronize()
    st0 = cloth.stats()
    cloth.set_kernel_timer(args.roofline_kernel)
    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    stream = torch.cuda.current_stream(dev)
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
    barrier(world)
    clk = clocks.stop()
    st1 = cloth.stats()
    cloth.set_kernel_timer("none")
    max_ms = aggregate(total_ms, world)
    value = world * args.steps * n_cloth / (max_ms / 1e3)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    x0h = x0.cpu().pin_memory()
    v0h = v0.cpu().pin_memory()
    xih = xi.cpu().pin_memory()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xN, vN = cloth.rollout(x0h, v0h, n_cloth)
        dx0, dv0, dth = cloth.backward(xih)
        _ = float(dth[0])
        e2e_s += time.perf_counter() - t0
    e2e_max = aggregate(e2e_s * 1e3, world) / 1e3
    m = sc.m
    e2e = {"value": world * args.steps * n_cloth / e2e_max, "unit": UNIT,
           "h2d_bytes_per_step": 3 * m * 3 * 8, "d2h_bytes_per_step": 4 * m * 3 * 8 + 3 * 8}

    # roofline of the dominant kernel (live CUDA-event timing over the timed region)
    launches = st1["timer_launches"]
    kern_ms = st1["timer_ms"] / max(launches, 1)
    if args.roofline_kernel == "front":
        n_fact = launches / max(st1["front_levels"], 1)
        work = st1["front_flops"] * n_fact / max(launches, 1)          # flops per launch (mean)
        achieved = work / (kern_ms / 1e3) / 1e12
        roof = {"kernel": "k_front_level (one level of the FP32 multifrontal LDL^T)", "bound": "alu",
                "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
        tr = TRAFFIC["front"]
        src = os.path.join(ROOT, "paper_2106_05306_gb300", "csrc", "dc_frontal.cu")
        roof["traffic"] = tr["bytes"] if tr["source_sha"] == kernel_sha(src) else None
    else:
        nnz = st1["fwd_solve_nnz"] if args.roofline_kernel == "solve_fwd" else st1["bwd_solve_nnz"]
        work = 6.0 * nnz                                                # 3 RHS FMAs per nonzero
        achieved = work / (kern_ms / 1e3) / 1e12
        roof = {"kernel": f"k_{args.roofline_kernel}", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "peak_source": "FP64 nominal 1.25 TFLOP/s",
                "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["mean_launch_us"] = kern_ms * 1e3
    roof["launches_timed"] = launches

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if n_cloth == N_STEPS else WORKLOAD.replace("125 steps", f"{n_cloth} steps"),
                   "cloth_steps_per_bench_step": n_cloth, "nodes": m,
                   "triangles": int(sc.tris.shape[0]), "pd_iters": p.n_pd_iters,
                   "checkpoint_every": CHECKPOINT_EVERY, "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MB write) before every timed step"},
        "e2e": e2e,
        "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
        "roofline": roof,
        "clocks": clk,
        "adjoint": {"gmres_iters_per_step": (st1["adj_iters"] - st0["adj_iters"]) / max(
            st1["adj_steps"] - st0["adj_steps"], 1), "nonconverged_steps": st1["adj_nonconverged"]},
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_subprocess()
    cloth.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    # each step: one bounded oracle sample of the workload (single-threaded child process)
    vals, secs = [], 0.0
    info = None
    for k in range(args.warmup + args.steps):
        info = cpu_baseline_subprocess()
        if k >= args.warmup:
            vals.append(info["value"])
            secs += info.get("seconds", 0.0)
    value = statistics.mean(vals) if vals and None not in vals else None
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": (1e3 / value) if value else None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": info["sample"] if info else None},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.cpu_sample:
        v, secs, sample = oracle_sample()
        print(json.dumps({"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                          "seconds": secs}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
