"""Benchmark: split-SART voxel-updates/s on the realistic slice, as one JSON line.

Workload: 512 x 128 voxels (N = 65536), K = 26 symmetric sources on +/-25 deg at
600 mm, 1024 detector bins (M = 26624), Siddon weights, a seeded 20-ellipse
phantom with 1% multiplicative Gaussian noise on p, 200 iterations, lambda = 0.8,
FP32.

One step is a reconstruction of the slice from its projections p:
- the device fold of A (folded CSR, CSC, normalisers) from the resident half
  rows;
- the fold of p;
- the persistent split-SART solve;
- the Theorem 1 recombination.

voxel-updates/s = N x iterations / step time. The L2 is flushed (256 MiB write)
between timed steps.

Arms:
- default (native): the CUDA library through the C ABI.
- ``--impl reference``: the CPU FP64 oracle, on the host cores, on the same
  workload.

Under torchrun each rank reconstructs its own slice (weak scaling, no
data-path collective). Rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "split-SART voxel-updates/s"
UNIT = "voxel-updates/s"
ITERS = 200
LAMBDA = 0.8
NOISE = 0.01
CONFIG_ID = 2
N_ELLIPSES = 20
PROFILE = os.path.join(ROOT, "profiles", "sart_persistent_realistic_fp32.txt")
KERNEL_SRC = os.path.join(ROOT, "paper_1902_10559_gb300", "csrc", "sart.cu")  # solve kernels


def workload_config(S=None):
    from paper_1902_10559_gb300.synthetic import REALISTIC as g
    cfg = {"workload": "realistic slice: 512x128 voxels, K=26 sources +/-25 deg, 1024 bins, 20 ellipses, 1% noise, "
                       "200 iterations, lambda=0.8, fp32",
           "nx": g.nx, "nz": g.nz, "N": g.N, "M": g.M, "iterations": ITERS, "lambda": LAMBDA,
           "l2": "flushed between timed steps (256 MiB write)"}
    if S is not None:
        cfg["S"] = S
    return cfg


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Sample nvidia-smi clocks and throttle reasons every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profile_traffic():
    """Per-launch DRAM bytes of the solve kernel from the committed ncu summary.

    Returns None if the summary is absent, or if the kernel source has changed
    since it was taken.
    """
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    src_hash = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_bytes or m_hash.group(1) != src_hash:
        return None
    return float(m_bytes.group(1))


def algorithmic_bytes_per_launch(S, Mh, Nh, iters):
    """Algorithmic bytes of one persistent FP32 solve.

    Forward pass (iters + 1 of them):
      12 S           col (4 B) and value pair (8 B) per entry
      4 (Mh + 1)     row pointers
      24 Mh          p pair read, 1/R pair read, u pair write
      8 Nh           f pairs, each gathered once
    Back pass (iters of them):
      12 S           row (4 B) and value pair (8 B) per entry
      4 (Nh + 1)     column pointers
      8 Mh           u pairs, each gathered once
      24 Nh          f pair read and write, 1/C pair read
    """
    fwd = 12 * S + 4 * (Mh + 1) + 24 * Mh + 8 * Nh
    bwd = 12 * S + 4 * (Nh + 1) + 8 * Mh + 24 * Nh
    return (iters + 1) * fwd + iters * bwd


def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1902_10559_gb300 import splitsart as ss
    from paper_1902_10559_gb300.synthetic import REALISTIC as g
    from paper_1902_10559_gb300.synthetic import apply_noise, noise_draws, random_phantom

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # Inputs: geometry (host Siddon), phantom, and projections p = A f (+1% noise).
    # Each rank reconstructs its own seeded slice.
    geom = ss.make_geometry(g)
    system = ss.fold_system(geom, ss.F32)
    info = system.info()
    img = random_phantom(g, CONFIG_ID, N_ELLIPSES, stream=10 * rank)
    f_img = torch.as_tensor(img.reshape(-1), dtype=torch.float32, device=dev)
    p = torch.empty(g.M, dtype=torch.float32, device=dev)
    ss.project(system, f_img, p, layout=ss.LAYOUT_IMAGE)
    eps = torch.as_tensor(noise_draws(g.M, CONFIG_ID, stream=10 * rank + 1), dtype=torch.float32, device=dev)
    p = (p * (1.0 + NOISE * eps)).contiguous()
    p12 = torch.empty(g.M // 2, 2, dtype=torch.float32, device=dev)
    f12 = torch.empty(g.N // 2, 2, dtype=torch.float32, device=dev)
    f = torch.empty(g.N, dtype=torch.float32, device=dev)
    opts = ss.solve_opts(ITERS, LAMBDA)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    n_launch = {"step": 0}

    def step(solve_events=None):
        ss.refold(system)                      # fold A: 5 kernels + 2 scans (3 kernels each)
        ss.fold_rhs(system, p, p12)            # 1 kernel
        f12.zero_()                            # f^0 = 0 (memset)
        if solve_events:
            solve_events[0].record(stream)
        ss.solve(system, p12, f12, opts)       # 1 persistent kernel
        if solve_events:
            solve_events[1].record(stream)
        ss.recombine(system, f12, f)           # 1 kernel
    n_launch["step"] = 5 + 2 * 3 + 1 + 1 + 1

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    res = ss.solve_result(system)
    iters = res["iters"]

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    s_solve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step(s_solve[k])
            ends[k].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    solve_ms = sum(a.elapsed_time(b) for a, b in s_solve) / args.steps
    res = ss.solve_result(system)

    # End to end through the public API with host buffers: pinned p in, image out.
    p_host = p.cpu().pin_memory()
    f_host = torch.empty(g.N, dtype=torch.float32).pin_memory()
    p_stage = torch.empty_like(p)

    def e2e_step():
        p_stage.copy_(p_host, non_blocking=True)
        ss.refold(system)
        ss.fold_rhs(system, p_stage, p12)
        f12.zero_()
        ss.solve(system, p12, f12, opts)
        ss.recombine(system, f12, f, layout=ss.LAYOUT_IMAGE)
        f_host.copy_(f, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    e_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        e_start[k].record(stream)
        e2e_step()
        e_end[k].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(s.elapsed_time(e) for s, e in zip(e_start, e_end))

    # Setup breakdown (untimed in the metric): refold alone.
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(0.0)
    a.record(stream)
    ss.refold(system)
    b.record(stream)
    torch.cuda.synchronize()
    fold_ms = a.elapsed_time(b)

    t_local = torch.tensor([step_ms, e2e_ms, solve_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    step_ms, e2e_ms, solve_ms = t_local.tolist()
    updates = g.N * iters * args.steps * ws
    value = updates / (step_ms / 1e3)
    e2e_value = updates / (e2e_ms / 1e3)

    S = info["S"]
    alg = algorithmic_bytes_per_launch(S, g.M // 2, g.N // 2, iters)
    peak, peak_kind = read_peaks()
    achieved = alg / (solve_ms / 1e3) / 1e9
    traffic = profile_traffic()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded random ellipses, Siddon projections, 1% noise)",
        "config": workload_config(S),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": g.M * 4, "d2h_bytes_per_step": g.N * 4},
        "gpu_launches": n_launch["step"] * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "sart_resident_kernel<TF32,8> (matrix slice kept in shared memory)",
                     "algorithmic_bytes_per_launch": alg, "peak_source": f"{peak_kind} hbm_gbs",
                     "note": "working set (~35 MB/iteration) is L2-resident within a solve"},
        "clocks": clocks.summary(),
        "breakdown_ms": {"solve": solve_ms, "fold_A": fold_ms, "step": step_ms / args.steps},
        "solve": {"iters": iters, "rho": res["rho"]},
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _oracle_workload():
    from oracle import geometry as ogeo
    from oracle import split as osplit
    from paper_1902_10559_gb300.synthetic import REALISTIC as g
    from paper_1902_10559_gb300.synthetic import apply_noise, noise_draws, random_phantom

    A = ogeo.mirrored_system_matrix(g)
    f_true = ogeo.image_to_snake(g, random_phantom(g, CONFIG_ID, N_ELLIPSES))
    p = apply_noise(A @ f_true, noise_draws(g.M, CONFIG_ID), NOISE)
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    return g, A1, A2, p1, p2


def cpu_baseline(budget_s: float):
    """Time the oracle split-SART on the same slice, on one host core.

    The sample is a bounded number of 200-iteration solves, as many as fit in
    about ``budget_s`` seconds (at least one).
    """
    from oracle import sart as osart
    g, A1, A2, p1, p2 = _oracle_workload()
    t0 = time.perf_counter()
    runs = 0
    while True:
        osart.split_sart(A1, A2, p1, p2, LAMBDA, ITERS)
        runs += 1
        el = time.perf_counter() - t0
        if el >= budget_s or runs >= 50:
            break
    value = g.N * ITERS * runs / el
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{runs} full 200-iteration FP64 solves of the same slice (SciPy CSR, single thread), "
                      f"{el:.1f} s; host has {os.cpu_count()} cores"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import sart as osart
    g, A1, A2, p1, p2 = _oracle_workload()
    for _ in range(args.warmup):
        osart.split_sart(A1, A2, p1, p2, LAMBDA, 20)  # short warm-up solves
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        osart.split_sart(A1, A2, p1, p2, LAMBDA, ITERS)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = g.N * ITERS * args.steps / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} full 200-iteration solves (SciPy CSR, single thread); "
                                      f"warm-up solves of 20 iterations; host has {os.cpu_count()} cores"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
