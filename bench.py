"""Benchmark of the symmetric-split SART path, printed as one JSON line.

Workloads (``--workload``):
- ``realistic`` (default): 512 x 128 voxels (N = 65536), K = 26 symmetric
  sources on +/-25 deg at 600 mm, 1024 detector bins (M = 26624), Siddon
  weights, a seeded 20-ellipse phantom with 1% multiplicative Gaussian noise
  on p, 200 iterations, lambda = 0.8, FP32.
- ``batch``: 256 independent slices of uneven size (nx in {256, 512, 768,
  1024}, nz in [64, 256], K in [16, 32], 2 nx bins), 200 iterations, lambda =
  0.8, FP32. The slices are solved in one persistent launch, replayed as a
  CUDA graph, with the launch shape chosen by the autotuner.
- ``multi``: 64 right-hand sides on the tiny slice's geometry (32 x 16 voxels,
  M = 640), 200 iterations, lambda = 0.8, FP32, solved as SpMM.

A step is one reconstruction of the workload from its projections p:
- the device fold of A (folded CSR, CSC, normalisers) from the resident half
  rows;
- the fold of p;
- the solve;
- the Theorem 1 recombination.
The metric is voxel-updates/s = (sum of N over slices and right-hand sides)
x iterations / step time. The L2 is flushed (256 MiB write) between timed
steps.

Arms:
- native (default): the CUDA library through the C ABI.
- ``--impl reference``: the CPU FP64 oracle, on the host cores, on a bounded
  sample of the same workload.

Under torchrun each rank reconstructs its own copy of the workload (weak
scaling, no data-path collective); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import ctypes
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
KERNEL_SRC = os.path.join(ROOT, "paper_1902_10559_gb300", "csrc", "sart.cu")  # solve kernels
PROFILES = os.path.join(ROOT, "profiles")
# Kernel launches of one device fold of A: count, scan (3), fill, row compaction (5),
# CSC count, scan (3), place, sort + column sums, column compaction (5).
FOLD_LAUNCHES = 21


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


def read_peak(key: str, fallback: float):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def profile_traffic(name: str):
    """Per-launch DRAM bytes of the solve kernel from a committed ncu summary.

    Returns None if the summary is absent, or if the kernel source has changed
    since it was taken.
    """
    try:
        txt = open(os.path.join(PROFILES, name)).read()
    except OSError:
        return None
    src_hash = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_bytes or m_hash.group(1) != src_hash:
        return None
    return float(m_bytes.group(1))


def algorithmic_bytes_per_launch(S, Mh, Nh, iters, batch_rows=0):
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
    A batch adds, per forward pass, 16 B per row: the per-row residual written
    and read back by its slice's stop test.
    """
    fwd = 12 * S + 4 * (Mh + 1) + 24 * Mh + 8 * Nh + 16 * batch_rows
    bwd = 12 * S + 4 * (Nh + 1) + 8 * Mh + 24 * Nh
    return (iters + 1) * fwd + iters * bwd


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def phantoms_projections(ss, system, geoms, dev, config_id, n_ell, rank, noise):
    """Seeded phantoms for every slice, projected on the device (+ noise). Returns p[M]."""
    import numpy as np
    import torch
    from paper_1902_10559_gb300.synthetic import noise_draws, random_phantom
    imgs = [random_phantom(g, config_id, n_ell, stream=1000 * rank + 2 * k) for k, g in enumerate(geoms)]
    f_img = torch.as_tensor(np.concatenate([im.reshape(-1) for im in imgs]), dtype=torch.float32, device=dev)
    p = torch.empty(system.M, dtype=torch.float32, device=dev)
    ss.project(system, f_img, p, layout=ss.LAYOUT_IMAGE)
    if noise:
        eps = np.concatenate([noise_draws(g.M, config_id, stream=1000 * rank + 2 * k + 1) for k, g in enumerate(geoms)])
        p = (p * (1.0 + noise * torch.as_tensor(eps, dtype=torch.float32, device=dev))).contiguous()
    return p


class Realistic:
    name = "realistic"
    config_id = 2
    profile = "sart_resident_realistic_fp32.txt"

    def setup(self, ss, dev, rank):
        import torch
        from paper_1902_10559_gb300 import autotune
        from paper_1902_10559_gb300.synthetic import REALISTIC as g
        self.g = g
        self.geoms = [g]
        self.geom = ss.make_geometry(g)
        self.system = ss.fold_system(self.geom, ss.F32)
        self.info = self.system.info()
        self.p = phantoms_projections(ss, self.system, [g], dev, self.config_id, 20, rank, NOISE)
        self.p12 = torch.empty(g.M // 2, 2, device=dev)
        self.f12 = torch.zeros(g.N // 2, 2, device=dev)
        self.f = torch.empty(g.N, device=dev)
        ss.fold_rhs(self.system, self.p, self.p12)
        self.tuned = autotune.tune_solve(self.system, self.p12, self.f12)
        self.opts = ss.solve_opts(ITERS, LAMBDA, **self.tuned)
        self.launches = FOLD_LAUNCHES + 3

    def step(self, ss, p_in, f_out, layout, ev=None):
        ss.refold(self.system)
        ss.fold_rhs(self.system, p_in, self.p12)
        self.f12.zero_()
        if ev:
            ev[0].record()
        ss.solve(self.system, self.p12, self.f12, self.opts)
        if ev:
            ev[1].record()
        ss.recombine(self.system, self.f12, f_out, layout=layout)

    def units(self, ss):
        return self.g.N * ss.solve_result(self.system)["iters"]

    def roofline(self, ss, solve_ms):
        S, Mh, Nh = self.info["S"], self.system.Mh, self.system.Nh
        alg = algorithmic_bytes_per_launch(S, Mh, Nh, ITERS)
        peak, kind = read_peak("hbm_gbs", 6800.0)
        ach = alg / (solve_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": profile_traffic(self.profile),
                "kernel": "sart_resident_kernel<TF32,LPC> (matrix slice kept in shared memory)"
                          if self.tuned.get("kernel") == 2 else "sart_stream_kernel<TF32,LPC>",
                "algorithmic_bytes_per_launch": alg, "peak_source": f"{kind} hbm_gbs",
                "note": "per-iteration working set ~35 MB is L2/shared-memory resident within a solve"}

    def config(self):
        return {"workload": "realistic slice: 512x128 voxels, K=26 sources +/-25 deg, 1024 bins, 20 ellipses, "
                            "1% noise, 200 iterations, lambda=0.8, fp32",
                "nx": self.g.nx, "nz": self.g.nz, "N": self.g.N, "M": self.g.M, "iterations": ITERS,
                "lambda": LAMBDA, "S": self.info["S"], "launch": self.tuned,
                "l2": "flushed between timed steps (256 MiB write)"}

    def oracle_case(self, budget_s):
        """Oracle inputs on the same slice (FP64, its own Siddon A)."""
        from oracle import geometry as ogeo
        from oracle import split as osplit
        from paper_1902_10559_gb300.synthetic import REALISTIC as g
        from paper_1902_10559_gb300.synthetic import apply_noise, noise_draws, random_phantom
        A = ogeo.mirrored_system_matrix(g)
        f_true = ogeo.image_to_snake(g, random_phantom(g, self.config_id, 20, stream=0))
        p = apply_noise(A @ f_true, noise_draws(g.M, self.config_id, stream=1), NOISE)
        A1, A2 = osplit.fold_matrix(A)
        p1, p2 = osplit.fold_rhs(p)
        return [(g.N, A1, A2, p1, p2)], "the full slice"


class Batch(Realistic):
    name = "batch"
    config_id = 3
    profile = "sart_stream_batch_fp32.txt"
    n_slices = 256

    def setup(self, ss, dev, rank):
        import torch
        from paper_1902_10559_gb300 import autotune
        from paper_1902_10559_gb300.synthetic import batch_geometries
        self.gs = batch_geometries()[: self.n_slices]
        self.geoms = [ss.make_geometry(g) for g in self.gs]
        self.system = ss.fold_batch(self.geoms, ss.F32)
        self.info = self.system.info()
        sysm = self.system
        self.p = phantoms_projections(ss, sysm, self.gs, dev, self.config_id, 12, rank, 0.0)
        self.p12 = torch.empty(sysm.Mh, 2, device=dev)
        self.f12 = torch.zeros(sysm.Nh, 2, device=dev)
        self.f = torch.empty(sysm.N, device=dev)
        ss.fold_rhs(sysm, self.p, self.p12)
        self.tuned = autotune.tune_solve(sysm, self.p12, self.f12, iters=3)
        self.opts = ss.solve_opts(ITERS, LAMBDA, **self.tuned)
        self.launches = FOLD_LAUNCHES + 3
        # The reconstruction after the fold of A, captured once as a CUDA graph and replayed per step.
        self.p_in = self.p
        self._run(ss)  # warm-up outside capture
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s), torch.cuda.graph(self.graph, stream=s):
            self._run(ss)
        torch.cuda.current_stream().wait_stream(s)

    def _run(self, ss):
        ss.fold_rhs(self.system, self.p_in, self.p12)
        self.f12.zero_()
        ss.solve(self.system, self.p12, self.f12, self.opts)
        ss.recombine(self.system, self.f12, self.f, layout=ss.LAYOUT_IMAGE)

    def step(self, ss, p_in, f_out, layout, ev=None):
        ss.refold(self.system)
        if p_in is not self.p_in:
            self.p_in.copy_(p_in, non_blocking=True)
        if ev:
            ev[0].record()
        self.graph.replay()
        if ev:
            ev[1].record()
        if f_out is not self.f:
            f_out.copy_(self.f, non_blocking=True)

    def units(self, ss):
        its = [i["iters"] for i in ss.solve_result_slices(self.system)]
        return sum(g.N * k for g, k in zip(self.gs, its))

    def roofline(self, ss, solve_ms):
        S, Mh, Nh = self.info["S"], self.system.Mh, self.system.Nh
        alg = algorithmic_bytes_per_launch(S, Mh, Nh, ITERS, batch_rows=Mh)
        # The timed graph also holds fold_rhs and recombine (about 0.1% of its bytes).
        peak, kind = read_peak("hbm_gbs", 6800.0)
        ach = alg / (solve_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": profile_traffic(self.profile), "kernel": "sart_stream_kernel<TF32,LPC,batch>",
                "algorithmic_bytes_per_launch": alg, "peak_source": f"{kind} hbm_gbs",
                "note": "timed region = the replayed graph (fold of p, solve, recombine); inputs far exceed L2"}

    def config(self):
        return {"workload": f"batch: {len(self.gs)} slices, nx in {{256,512,768,1024}}, nz in [64,256], K in [16,32], "
                            "nb=2nx, 200 iterations, lambda=0.8, fp32, one persistent launch in a CUDA graph",
                "slices": len(self.gs), "N": self.system.N, "M": self.system.M, "S": self.info["S"],
                "iterations": ITERS, "lambda": LAMBDA, "launch": self.tuned,
                "l2": "inputs larger than L2 (about 10 GB per iteration), L2 also flushed between steps"}

    def oracle_case(self, budget_s):
        from oracle import geometry as ogeo
        from oracle import split as osplit
        from paper_1902_10559_gb300.synthetic import batch_geometries, random_phantom
        gs = batch_geometries()
        order = sorted(range(len(gs)), key=lambda k: gs[k].N)[:4]
        cases = []
        for k in order:
            g = gs[k]
            A = ogeo.mirrored_system_matrix(g)
            f_true = ogeo.image_to_snake(g, random_phantom(g, self.config_id, 12, stream=2 * k))
            A1, A2 = osplit.fold_matrix(A)
            p1, p2 = osplit.fold_rhs(A @ f_true)
            cases.append((g.N, A1, A2, p1, p2))
        return cases, "the 4 smallest slices of the batch"


class Multi(Realistic):
    name = "multi"
    config_id = 3
    profile = "sart_multi_tiny64_fp32.txt"
    NRHS = 64

    def setup(self, ss, dev, rank):
        import torch
        from paper_1902_10559_gb300 import autotune
        from paper_1902_10559_gb300.synthetic import TINY
        self.g = TINY
        self.geom = ss.make_geometry(TINY)
        self.system = ss.fold_system(self.geom, ss.F32)
        self.info = self.system.info()
        # A batch of NRHS copies of the slice gives the [nrhs][M] and [nrhs][Mh] layouts of
        # solve_multi, so p is folded and f recombined for all right-hand sides in one launch each.
        self.vec = ss.fold_batch([self.geom] * self.NRHS, ss.F32)
        self.p = phantoms_projections(ss, self.vec, [TINY] * self.NRHS, dev, self.config_id, 8, rank, 0.0)
        self.p12 = torch.empty(self.NRHS, TINY.M // 2, 2, device=dev)
        self.f12 = torch.zeros(self.NRHS, TINY.N // 2, 2, device=dev)
        self.f = torch.empty(self.NRHS * TINY.N, device=dev)
        self.infobuf = torch.zeros(self.NRHS * ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device=dev)
        ss.fold_rhs(self.vec, self.p, self.p12.view(-1, 2))
        self.tuned = autotune.tune_multi(self.system, self.p12, self.f12)
        self.opts = ss.solve_opts(ITERS, LAMBDA, block_threads=self.tuned["block_threads"])
        self.launches = FOLD_LAUNCHES + 3

    def step(self, ss, p_in, f_out, layout, ev=None):
        ss.refold(self.system)
        ss.fold_rhs(self.vec, p_in, self.p12.view(-1, 2))
        self.f12.zero_()
        if ev:
            ev[0].record()
        ss.solve_multi(self.system, self.p12, self.f12, self.opts, self.infobuf,
                       rhs_per_cta=self.tuned["rhs_per_cta"])
        if ev:
            ev[1].record()
        ss.recombine(self.vec, self.f12.view(-1, 2), f_out, layout=layout)

    def units(self, ss):
        return sum(self.g.N * i["iters"] for i in ss.read_infos(self.infobuf, self.NRHS))

    def roofline(self, ss, solve_ms):
        S = self.info["S"]
        flops = 8.0 * S * self.NRHS * ITERS  # 2 systems x FMA x (forward + back)
        # FP32 CUDA-core FMA peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz.
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        ach = flops / (solve_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": profile_traffic(self.profile), "kernel": "sart_multi_kernel<TF32,RC>",
                "peak_source": "nominal FP32 FMA rate at 2.07 GHz",
                "note": "system and vectors in shared memory; latency- and shared-memory-bound, not DRAM"}

    def config(self):
        return {"workload": "64 right-hand sides on the tiny slice geometry (32x16 voxels, M=640), 200 iterations, "
                            "lambda=0.8, fp32, SpMM", "nrhs": self.NRHS, "N": self.g.N, "M": self.g.M,
                "S": self.info["S"], "iterations": ITERS, "launch": self.tuned,
                "l2": "flushed between timed steps (256 MiB write)"}

    def oracle_case(self, budget_s):
        from oracle import geometry as ogeo
        from oracle import split as osplit
        from paper_1902_10559_gb300.synthetic import TINY, random_phantom
        A = ogeo.mirrored_system_matrix(TINY)
        A1, A2 = osplit.fold_matrix(A)
        cases = []
        for r in range(self.NRHS):
            f_true = ogeo.image_to_snake(TINY, random_phantom(TINY, self.config_id, 8, stream=2 * r))
            p1, p2 = osplit.fold_rhs(A @ f_true)
            cases.append((TINY.N, A1, A2, p1, p2))
        return cases, "all 64 right-hand sides"


WORKLOADS = {"realistic": Realistic, "batch": Batch, "multi": Multi}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def oracle_throughput(wl, budget_s):
    """Oracle voxel-updates/s on a bounded sample of the workload (single thread)."""
    from oracle import sart as osart
    cases, what = wl.oracle_case(budget_s)
    t0 = time.perf_counter()
    done = 0
    units = 0
    while True:
        for n, A1, A2, p1, p2 in cases:
            osart.split_sart(A1, A2, p1, p2, LAMBDA, ITERS)
            units += n * ITERS
            done += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return units / el, {"value": units / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                        "sample": f"{done} full {ITERS}-iteration FP64 solves from {what} (SciPy CSR, single "
                                  f"thread), {el:.1f} s; host has {os.cpu_count()} cores"}


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_1902_10559_gb300 import splitsart as ss

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    wl = WORKLOADS[args.workload]()
    wl.setup(ss, dev, rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        wl.step(ss, wl.p, wl.f, ss.LAYOUT_IMAGE)
    torch.cuda.synchronize()

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
            wl.step(ss, wl.p, wl.f, ss.LAYOUT_IMAGE, s_solve[k])
            ends[k].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    solve_ms = sum(a.elapsed_time(b) for a, b in s_solve) / args.steps
    units = wl.units(ss)

    # End to end through the public API with host buffers: pinned p in, image out.
    p_host = wl.p.cpu().pin_memory()
    f_host = torch.empty(wl.f.numel(), dtype=torch.float32).pin_memory()
    p_stage = torch.empty_like(wl.p)
    f_stage = torch.empty_like(wl.f)

    def e2e_step():
        p_stage.copy_(p_host, non_blocking=True)
        wl.step(ss, p_stage, f_stage, ss.LAYOUT_IMAGE)
        f_host.copy_(f_stage, non_blocking=True)

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

    # Fold of A alone (part of every step).
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(0.0)
    a.record(stream)
    ss.refold(wl.system)
    b.record(stream)
    torch.cuda.synchronize()
    fold_ms = a.elapsed_time(b)

    t_local = torch.tensor([step_ms, e2e_ms, solve_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    step_ms, e2e_ms, solve_ms = t_local.tolist()
    total_units = units * args.steps * ws
    value = total_units / (step_ms / 1e3)
    e2e_value = total_units / (e2e_ms / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded random ellipses, Siddon projections)",
        "config": wl.config(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": wl.p.numel() * 4,
                "d2h_bytes_per_step": wl.f.numel() * 4},
        "gpu_launches": wl.launches * args.steps,
        "roofline": wl.roofline(ss, solve_ms),
        "clocks": clocks.summary(),
        "breakdown_ms": {"solve": solve_ms, "fold_A": fold_ms, "step": step_ms / args.steps},
    }
    if rank == 0 and not args.no_cpu_baseline:
        _, out["cpu_baseline"] = oracle_throughput(wl, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import sart as osart
    wl = WORKLOADS[args.workload]()
    cases, what = wl.oracle_case(0)
    for _ in range(args.warmup):
        n, A1, A2, p1, p2 = cases[0]
        osart.split_sart(A1, A2, p1, p2, LAMBDA, 5)  # short warm-up solves
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        for n, A1, A2, p1, p2 in cases:
            osart.split_sart(A1, A2, p1, p2, LAMBDA, ITERS)
            units += n * ITERS
    total = time.perf_counter() - t0
    value = units / total
    cfg = {"workload": f"oracle on {what} of the {args.workload} workload", "iterations": ITERS, "lambda": LAMBDA}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} x {what}, full {ITERS}-iteration solves (SciPy CSR, single "
                                      f"thread); host has {os.cpu_count()} cores"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="realistic")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--slices", type=int, default=256, help="batch workload: number of slices (first n of the 256)")
    args = ap.parse_args()
    Batch.n_slices = max(1, min(256, args.slices))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
