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
KERNEL_SRC = os.path.join(ROOT, "paper_1902_10559_gb300", "csrc", "sart.cu")  # solve kernels 1-4
STREAM_SRC = os.path.join(ROOT, "paper_1902_10559_gb300", "csrc", "stream.cu")  # solve kernels 5 and 6
RING_SRC = os.path.join(ROOT, "paper_1902_10559_gb300", "csrc", "ring.cu")  # solve kernels 7 and 8
MULTI_SRC = os.path.join(ROOT, "paper_1902_10559_gb300", "csrc", "multi.cu")  # multi-RHS solve kernel
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


def profile_traffic(name: str, src: str = KERNEL_SRC, algorithmic_bytes: float | None = None,
                    ratio_key: str = "dram_over_algorithmic"):
    """Per-launch DRAM bytes of the solve kernel from a committed ncu summary.

    A summary gives either ``dram_bytes_per_launch`` (captured on the bench's
    own launch) or ``dram_over_algorithmic`` (captured on a smaller case of the
    same kernel whose traffic grows with its algorithmic bytes; it is then
    scaled by ``algorithmic_bytes``, the bench launch's).
    Returns None if the summary is absent, or if the kernel's source file
    (``src``) has changed since it was taken.
    """
    try:
        txt = open(os.path.join(PROFILES, name)).read()
    except OSError:
        return None
    src_hash = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m_hash or m_hash.group(1) != src_hash:
        return None
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if m_bytes:
        return float(m_bytes.group(1))
    m_ratio = re.search(re.escape(ratio_key) + r":\s*([0-9.eE+]+)", txt)
    if m_ratio and algorithmic_bytes:
        return float(m_ratio.group(1)) * algorithmic_bytes
    return None


def algorithmic_bytes_per_launch(S, Mh, Nh, iters, batch_rows=0, bytes_per_entry=12):
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
    The implicit fold stores each half-row entry once (4 B index with the sign,
    4 B length): bytes_per_entry = 8 with S = the half rows' entries.
    """
    fwd = bytes_per_entry * S + 4 * (Mh + 1) + 24 * Mh + 8 * Nh + 16 * batch_rows
    bwd = bytes_per_entry * S + 4 * (Nh + 1) + 8 * Mh + 24 * Nh
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
    default_steps = 100  # about 0.26 s of timed steps
    iters = ITERS
    lam = LAMBDA
    metric, unit, higher_is_better, dtype = METRIC, UNIT, True, "f32"
    two_process_baseline = True  # also time the oracle with A1 and A2 in two processes

    def oracle_run(self, osart, case):
        """One oracle solve of a sampled case; returns the units it completed."""
        n, A1, A2, p1, p2 = case
        osart.split_sart(A1, A2, p1, p2, self.lam, self.iters)
        return n * self.iters

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
        self.opts = ss.solve_opts(self.iters, self.lam, **self.tuned)
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
        alg = algorithmic_bytes_per_launch(S, Mh, Nh, self.iters)
        peak, kind = read_peak("hbm_gbs", 6800.0)
        ach = alg / (solve_ms / 1e3) / 1e9
        traffic = profile_traffic(self.profile)
        out = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
               "traffic": traffic,
               "kernel": "sart_resident_kernel<TF32,LPC> (matrix slice kept in shared memory)"
                         if self.tuned.get("kernel") == 2 else "sart_stream_kernel<TF32,LPC>",
               "algorithmic_bytes_per_launch": alg, "peak_source": f"{kind} hbm_gbs",
               "achieved_is": "effective bandwidth: algorithmic bytes of the solve / solve time. The per-iteration "
                              "working set (about 35 MB) stays in shared memory and L2, so this is not DRAM "
                              "traffic; dram_gbs is"}
        if traffic:
            out["dram_gbs"] = traffic / (solve_ms / 1e3) / 1e9
            out["dram_frac"] = out["dram_gbs"] / peak
        out["on_chip"] = self.latency_floor(ss, solve_ms)
        return out

    def latency_floor(self, ss, solve_ms):
        """The resident kernel's latency bound, measured.

        The same kernel and launch shape on the tiny slice (S = 3,394 entries over
        152 CTAs: a few rows and columns each) runs every per-iteration step that
        does not scale with the matrix: the two grid barriers, the norm reduction,
        the stop test, and one round of dependent gathers each way. Its time per
        iteration is the floor under this kernel; frac = floor / the realistic
        slice's time per iteration.
        """
        import torch
        from paper_1902_10559_gb300.synthetic import TINY
        if self.tuned.get("kernel") != 2:
            return None
        tiny = ss.fold_system(ss.make_geometry(TINY), ss.F32)
        p12 = torch.zeros(TINY.M // 2, 2, device=self.p12.device)
        p12[:, 1] = 1.0
        f12 = torch.zeros(TINY.N // 2, 2, device=self.p12.device)
        ts = []
        for _ in range(4):
            f12.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ss.solve(tiny, p12, f12, self.opts)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        floor_us = min(ts[1:]) * 1e3 / self.iters
        per_us = solve_ms * 1e3 / self.iters
        return {"bound": "latency", "floor_us_per_iteration": floor_us, "us_per_iteration": per_us,
                "frac": floor_us / per_us,
                "floor_from": "the same kernel and launch shape on the tiny slice (3,394 entries): two grid barriers "
                              "and one round of dependent gathers each way per iteration (with tol = 0, as here, "
                              "rho is tested at the first and the last iteration only)"}

    def extra(self, ss):
        """Workload-specific keys added to the JSON line."""
        return {"forms": self.form_times(ss, [self.geom])}

    def form_times(self, ss, geoms):
        """Solve time of the same inputs with BF16 and FP16 matrix values (per-row scales), beside FP32."""
        import torch
        out = {}
        ts32 = None
        for name, dt in (("f32", ss.F32), ("bf16", ss.BF16), ("f16", ss.F16)):
            sysm = self.system if dt == ss.F32 else (
                ss.fold_system(geoms[0], dt) if len(geoms) == 1 else ss.fold_batch(geoms, dt))
            p12 = torch.empty(sysm.Mh, 2, device=self.p12.device)
            ss.fold_rhs(sysm, self.p_in if hasattr(self, "p_in") else self.p, p12)
            f12 = torch.zeros(sysm.Nh, 2, device=self.p12.device)
            ts = []
            for _ in range(3):
                f12.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ss.solve(sysm, p12, f12, self.opts)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            out[name] = {"solve_ms": min(ts[1:]), "bytes_per_entry_per_pass": 12 if dt == ss.F32 else 8}
            if dt != ss.F32:
                out[name]["time_vs_f32"] = out[name]["solve_ms"] / out["f32"]["solve_ms"]
                del sysm
                torch.cuda.empty_cache()
        out["note"] = "same inputs, launch shape and iterations as the timed FP32 solve"
        return out

    def config(self):
        return {"workload": "realistic slice: 512x128 voxels, K=26 sources +/-25 deg, 1024 bins, 20 ellipses, "
                            "1% noise, 200 iterations, lambda=0.8, fp32",
                "nx": self.g.nx, "nz": self.g.nz, "N": self.g.N, "M": self.g.M, "iterations": self.iters,
                "lambda": self.lam, "S": self.info["S"], "launch": self.tuned,
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
    two_process_baseline = False
    config_id = 3
    profile = "sart_rows_batch_fp32.txt"
    default_steps = 10
    n_slices = 256

    def setup(self, ss, dev, rank):
        import torch
        from paper_1902_10559_gb300 import autotune
        from paper_1902_10559_gb300.synthetic import batch_geometries
        from paper_1902_10559_gb300.synthetic import TINY
        self.gs = batch_geometries()[: self.n_slices]
        ss.make_geometries_device([TINY])  # loads the tracer's kernels
        t0 = time.perf_counter()
        self.geoms = ss.make_geometries_device(self.gs)
        t1 = time.perf_counter()
        self.system = ss.fold_batch(self.geoms, ss.F32)
        torch.cuda.synchronize()
        self.geometry_s = {"device_tracer": t1 - t0, "device_tracer_and_fold": time.perf_counter() - t0}
        self.info = self.system.info()
        sysm = self.system
        self.p = phantoms_projections(ss, sysm, self.gs, dev, self.config_id, 12, rank, 0.0)
        self.p12 = torch.empty(sysm.Mh, 2, device=dev)
        self.f12 = torch.zeros(sysm.Nh, 2, device=dev)
        self.f = torch.empty(sysm.N, device=dev)
        ss.fold_rhs(sysm, self.p, self.p12)
        self.tuned = autotune.tune_solve(sysm, self.p12, self.f12, iters=3)
        self.opts = ss.solve_opts(self.iters, self.lam, **self.tuned)
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
        alg = algorithmic_bytes_per_launch(S, Mh, Nh, self.iters, batch_rows=Mh)
        # The timed graph also holds fold_rhs and recombine (about 0.1% of its bytes).
        peak, kind = read_peak("hbm_gbs", 6800.0)
        ach = alg / (solve_ms / 1e3) / 1e9
        traffic = self.traffic(self.tuned.get("kernel"), alg)
        out = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
               "traffic": traffic, "kernel": self.kernel_name(),
               "algorithmic_bytes_per_launch": alg, "peak_source": f"{kind} hbm_gbs",
               "traffic_source": "ncu DRAM counters of the same kernel on the 64-slice case (one launch), scaled to "
                                 "this launch by algorithmic bytes",
               "note": "timed region = the replayed graph (fold of p, solve, recombine); inputs far exceed L2"}
        if traffic:
            out["dram_gbs"] = traffic / (solve_ms / 1e3) / 1e9
            out["dram_frac"] = out["dram_gbs"] / peak
        return out

    def extra(self, ss, host_tracer=True):
        # Setup, outside the timed steps: the first-half rows of all slices
        # traced on the GPU, and (host_tracer) on the host cores for comparison.
        import torch
        if host_tracer:
            t0 = time.perf_counter()
            host = [ss.make_geometry(g) for g in self.gs]
            t1 = time.perf_counter()
            sysm = ss.fold_batch(host, ss.F32)
            torch.cuda.synchronize()
            self.geometry_s["host_tracer"] = t1 - t0
            self.geometry_s["host_tracer_and_fold"] = time.perf_counter() - t0
            self.geometry_s["host_threads"] = min(32, os.cpu_count() or 1)
            del host, sysm
        return {"forms": self.form_times(ss, self.geoms), "geometry_s": self.geometry_s}

    def traffic(self, kernel, alg):
        """DRAM bytes of one launch of `kernel`, from the committed 64-slice capture of that kernel."""
        if kernel == 5:
            return profile_traffic("sart_compact_batch_fp32.txt", STREAM_SRC, alg)
        if kernel == 6:
            return profile_traffic("sart_compact_batch_fp32.txt", STREAM_SRC, alg, "dram_over_algorithmic_implicit")
        if kernel == 7:
            return profile_traffic("sart_ring_batch_fp32.txt", RING_SRC, alg)
        if kernel == 8:
            return profile_traffic("sart_ring_batch_fp32.txt", RING_SRC, alg, "dram_over_algorithmic_implicit")
        if kernel == 3:
            return profile_traffic(self.profile, KERNEL_SRC, alg)
        return None

    def form_times(self, ss, geoms):
        """Solve time of the same inputs in each storage form and kernel, each with its own roofline.

        f32: the timed solve (autotuned launch shape). f32_rows: the row-streaming
        kernel (3). f32_compact: the compacted-order kernel (5) on the explicit
        fold. f32_implicit: kernel 5's design on the implicit fold (6), 8 bytes
        per half-row entry and pass. f32_ring / f32_ring_implicit: the same two
        folds fed through a producer warp's shared-memory ring (kernels 7 and 8).
        bf16 / f16: 2-byte codes with per-row scales (8 bytes per entry and pass)
        on the row-streaming kernel; *_compact: the same codes on kernel 5;
        bf16_ring: on kernel 7.
        """
        import torch
        peak, _ = read_peak("hbm_gbs", 6800.0)
        S, Mh, Nh = self.info["S"], self.system.Mh, self.system.Nh
        nnz_half = self.info["nnz_half"]
        lpc = self.tuned.get("lanes_per_col", 4) or 4
        forms = [("f32", ss.F32, self.opts, 12, S),
                 ("f32_rows", ss.F32, ss.solve_opts(self.iters, self.lam, kernel=3, lanes_per_col=lpc,
                                                    block_threads=512), 12, S),
                 ("f32_compact", ss.F32, ss.solve_opts(self.iters, self.lam, kernel=5, lanes_per_col=4,
                                                       block_threads=512), 12, S),
                 ("f32_implicit", ss.F32, ss.solve_opts(self.iters, self.lam, kernel=6, lanes_per_col=4,
                                                        block_threads=512), 8, nnz_half),
                 ("f32_ring", ss.F32, ss.solve_opts(self.iters, self.lam, kernel=7, lanes_per_col=4), 12, S),
                 ("f32_ring_implicit", ss.F32, ss.solve_opts(self.iters, self.lam, kernel=8, lanes_per_col=4), 8,
                  nnz_half),
                 ("bf16", ss.BF16, ss.solve_opts(self.iters, self.lam, kernel=3, lanes_per_col=lpc,
                                                 block_threads=512), 8, S),
                 ("bf16_compact", ss.BF16, ss.solve_opts(self.iters, self.lam, kernel=5, lanes_per_col=4,
                                                         block_threads=512), 8, S),
                 ("bf16_ring", ss.BF16, ss.solve_opts(self.iters, self.lam, kernel=7, lanes_per_col=4), 8, S),
                 ("f16", ss.F16, ss.solve_opts(self.iters, self.lam, kernel=3, lanes_per_col=lpc,
                                                block_threads=512), 8, S),
                 ("f16_compact", ss.F16, ss.solve_opts(self.iters, self.lam, kernel=5, lanes_per_col=4,
                                                        block_threads=512), 8, S)]
        out = {}
        reduced = {}
        for name, dt, opts, bpe, entries in forms:
            if dt != ss.F32 and dt not in reduced:
                reduced.clear()
                torch.cuda.empty_cache()
                reduced[dt] = ss.fold_batch(geoms, dt)
            sysm = self.system if dt == ss.F32 else reduced[dt]
            p12 = torch.empty(sysm.Mh, 2, device=self.p12.device)
            ss.fold_rhs(sysm, self.p_in, p12)
            f12 = torch.zeros(sysm.Nh, 2, device=self.p12.device)
            ts = []
            for _ in range(3):
                f12.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ss.solve(sysm, p12, f12, opts)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            ms = min(ts[1:])
            alg = algorithmic_bytes_per_launch(entries, Mh, Nh, self.iters, batch_rows=Mh, bytes_per_entry=bpe)
            out[name] = {"solve_ms": ms, "kernel": opts.kernel, "bytes_per_entry_per_pass": bpe,
                         "algorithmic_bytes_per_launch": alg, "hbm_frac": alg / (ms / 1e3) / 1e9 / peak,
                         "time_vs_f32_rows": None}
            tr = self.traffic(opts.kernel, alg) if dt == ss.F32 else None
            if tr:
                out[name]["dram_frac"] = tr / (ms / 1e3) / 1e9 / peak
            del sysm
        reduced.clear()
        torch.cuda.empty_cache()
        for name in out:
            out[name]["time_vs_f32_rows"] = out[name]["solve_ms"] / out["f32_rows"]["solve_ms"]
        out["note"] = ("same inputs and iterations; hbm_frac = each form's own algorithmic bytes / solve time / "
                       "measured HBM peak")
        return out

    def kernel_name(self):
        return {1: "sart_stream_kernel<TF32,LPC,batch> (CTA-wide staged tiles)",
                2: "sart_resident_kernel<TF32,LPC>",
                3: "sart_rows_kernel<TF32,LPC,batch> (row streaming, dynamically scheduled chunks)",
                4: "sart_bulk_kernel<TF32,LPC,batch> (per-warp bulk-copy staging)",
                5: "sart_compact_kernel<TF32,explicit,batch> (row streaming in compacted index order)",
                6: "sart_compact_kernel<TF32,implicit,batch> (row streaming in compacted index order)",
                7: "sart_ring_kernel<TF32,explicit,batch> (compacted order through a producer warp's ring)",
                8: "sart_ring_kernel<TF32,implicit,batch> (compacted order through a producer warp's ring)"}.get(
            self.tuned.get("kernel"), "sart_rows_kernel<TF32,LPC,batch> (library choice)")

    def config(self):
        return {"workload": f"batch: {len(self.gs)} slices, nx in {{256,512,768,1024}}, nz in [64,256], K in [16,32], "
                            "nb=2nx, 200 iterations, lambda=0.8, fp32, one persistent launch in a CUDA graph",
                "slices": len(self.gs), "N": self.system.N, "M": self.system.M, "S": self.info["S"],
                "iterations": self.iters, "lambda": self.lam, "launch": self.tuned,
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
    two_process_baseline = False

    def extra(self, ss):
        return {}
    config_id = 3
    profile = "sart_multi_tiny64_fp32.txt"
    default_steps = 200
    NRHS = 64
    ktype = "TF32"

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
        self.opts = ss.solve_opts(self.iters, self.lam, block_threads=self.tuned["block_threads"],
                                  lanes_per_row=self.tuned.get("lanes_per_row", 0))
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
        flops = 8.0 * S * self.NRHS * self.iters  # 2 systems x FMA x (forward + back)
        # FP32 CUDA-core FMA peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz.
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        ach = flops / (solve_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": profile_traffic(self.profile, MULTI_SRC), "kernel": f"sart_multi_kernel<{self.ktype},RC>",
                "peak_source": "nominal FP32 FMA rate at 2.07 GHz",
                "note": "system and vectors in shared memory; latency- and shared-memory-bound, not DRAM"}

    def config(self):
        return {"workload": "64 right-hand sides on the tiny slice geometry (32x16 voxels, M=640), 200 iterations, "
                            "lambda=0.8, fp32, SpMM", "nrhs": self.NRHS, "N": self.g.N, "M": self.g.M,
                "S": self.info["S"], "iterations": self.iters, "launch": self.tuned,
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


class Precision(Multi):
    """Matrix values stored as BF16 (timed) and FP16, with per-row FP32 scales.

    The step is the 64-right-hand-side tiny-slice SpMM for 500 iterations,
    lambda = 1, with BF16 values. The line adds, for FP32, BF16 and FP16
    storage, the iterations and time to rho <= 1e-3, and each reduced form's
    distance from the FP32 result after 500 iterations. Errors against the
    FP64 oracle are checked in the precision tests.
    """
    name = "precision"
    config_id = 4
    profile = "sart_multi_tiny64_bf16.txt"
    default_steps = 100
    iters = 500
    lam = 1.0
    ktype = "TBF16"
    dtype = "bf16 values, f32 accumulation"
    TOL = 1e-3
    MAX_ITERS = 30000

    def setup(self, ss, dev, rank):
        from paper_1902_10559_gb300 import autotune
        super().setup(ss, dev, rank)
        self.forms = {"f32": (self.system, self.tuned),
                      "bf16": (ss.fold_system(self.geom, ss.BF16), None),
                      "f16": (ss.fold_system(self.geom, ss.F16), None)}
        for k in ("bf16", "f16"):
            sysm = self.forms[k][0]
            self.forms[k] = (sysm, autotune.tune_multi(sysm, self.p12, self.f12))
        self.system, self.tuned = self.forms["bf16"]
        self.info = self.system.info()
        self.opts = ss.solve_opts(self.iters, self.lam, block_threads=self.tuned["block_threads"])

    def time_to_tol(self, ss):
        """Per storage form: the launch time and iterations of the 64 right-hand sides to rho <= 1e-3."""
        import numpy as np
        import torch
        out = {}
        for name, (sysm, tuned) in self.forms.items():
            f12 = torch.zeros_like(self.f12)
            opts = ss.solve_opts(self.MAX_ITERS, self.lam, self.TOL, block_threads=tuned["block_threads"],
                                 lanes_per_row=tuned.get("lanes_per_row", 0))
            ts = []
            for _ in range(3):
                f12.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ss.solve_multi(sysm, self.p12, f12, opts, self.infobuf, rhs_per_cta=tuned["rhs_per_cta"])
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            infos = ss.read_infos(self.infobuf, self.NRHS)
            its = np.array([i["iters"] for i in infos])
            reached = np.array([i["rho"] <= self.TOL for i in infos])
            out[name] = {"ms": float(np.median(ts)), "iters_mean": float(its.mean()), "iters_max": int(its.max()),
                         "reached": float(reached.mean()), "launch": tuned}
        for name in ("bf16", "f16"):
            out[name]["time_vs_plain_f32"] = out[name]["ms"] / out["f32"]["ms"]
        return out

    def extra(self, ss):
        import torch
        out = self.time_to_tol(ss)
        finals = {}
        for name, (sysm, tuned) in self.forms.items():
            # 500 iterations, for the distance between forms.
            f12 = torch.zeros_like(self.f12)
            ss.solve_multi(sysm, self.p12, f12, ss.solve_opts(self.iters, self.lam,
                                                              block_threads=tuned["block_threads"],
                                                              lanes_per_row=tuned.get("lanes_per_row", 0)),
                           self.infobuf, rhs_per_cta=tuned["rhs_per_cta"])
            img = torch.empty(self.NRHS * self.g.N, device=f12.device)
            ss.recombine(self.vec, f12.view(-1, 2), img, layout=ss.LAYOUT_IMAGE)
            finals[name] = img.double()
        for name in ("bf16", "f16"):
            d = torch.linalg.vector_norm(finals[name] - finals["f32"]) / torch.linalg.vector_norm(finals["f32"])
            out[name]["rel_diff_vs_f32_at_500"] = float(d)
        return {"time_to_rho_1e-3": out,
                "note": "64 right-hand sides, one solve_multi launch each; ms is the launch time until the last "
                        "right-hand side stops; errors against the FP64 oracle are in the precision tests"}

    def config(self):
        c = super().config()
        c["workload"] = ("64 right-hand sides on the tiny slice geometry (32x16 voxels, M=640), 500 iterations, "
                         "lambda=1, BF16 matrix values with per-row FP32 scales, FP32 accumulation, SpMM")
        return c


class Warmstart(Multi):
    """Learned warm start against plain split-SART, both to rho <= 1e-3.

    Setup: 20000 seeded training phantoms on the tiny slice geometry; inputs
    are the 5-iteration images and targets the 500-iteration images, all made
    by the library's solver; the network is trained with the library's
    kernels (Adam, batch 64). The step reconstructs 512 held-out phantoms
    (seeds 10^6 + k) to rho <= 1e-3: 5 iterations, network, fold of the
    image, fallback test, then split-SART to the tolerance, and the Theorem 1
    recombination. The line adds the plain solve of the same 512 from zero.
    """
    name = "warmstart"
    config_id = 5
    profile = "sart_multi_tiny64_fp32.txt"
    default_steps = 5
    iters = 30000  # iteration cap
    lam = 1.0
    metric = "split-SART reconstructions to relative residual 1e-3 per second"
    unit = "reconstructions/s"
    dtype = "f32 solve, bf16 tensor-core convolutions"
    TOL = 1e-3
    N_TRAIN = 20000
    N_HELD = 512
    EPOCHS = 6

    def setup(self, ss, dev, rank):
        import numpy as np
        import torch
        from paper_1902_10559_gb300.synthetic import TINY
        from paper_1902_10559_gb300.warmstart import WarmStart
        self.g = TINY
        self.ws = WarmStart(TINY, lam=self.lam)
        self.system = self.ws.system
        self.info = self.system.info()
        t0 = time.perf_counter()
        x, t = self.ws.make_pairs(np.arange(self.N_TRAIN))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        self.loss_hist = self.ws.train(x, t, epochs=self.EPOCHS, batch=64, lr=1e-3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        self.setup_s = {"training_pairs": t1 - t0, "training": t2 - t1}
        del x, t
        held = np.arange(10 ** 6, 10 ** 6 + self.N_HELD)
        self.p = self.ws.project(self.ws.phantoms(held)).reshape(-1).contiguous()
        self.f = torch.empty(self.N_HELD * TINY.N, device=dev)
        self.launches = 0  # counted per step below
        self._infos = None

    def step(self, ss, p_in, f_out, layout, ev=None):
        ss.refold(self.system)
        p12 = self.ws.fold_rhs(p_in.view(self.N_HELD, -1))
        if ev:
            ev[0].record()
        f12, e, r, picked = self.ws.solve_warm(p12, self.TOL, self.iters)
        if ev:
            ev[1].record()
        self._infos = (e, r)
        f_out.view(self.N_HELD, -1).copy_(self.ws.recombine(f12).view(self.N_HELD, -1))

    def units(self, ss):
        return self.N_HELD

    def _counts(self, ss):
        e, r = self._infos
        return self.ws.warm_counts(ss.read_infos(e, self.N_HELD), ss.read_infos(r, self.N_HELD), self.TOL)

    def roofline(self, ss, solve_ms):
        its, _ = self._counts(ss)
        flops = 8.0 * self.info["S"] * float(its.sum())
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        ach = flops / (solve_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "sart_multi_kernel<TF32,RC> (the solves dominate the warm pipeline)",
                "peak_source": "nominal FP32 FMA rate at 2.07 GHz",
                "note": "useful FMAs of the iterations each right-hand side needed, over the whole warm pipeline"}

    def time_to_tol(self, ss):
        """The warm pipeline and the plain solve of the 512 held-out right-hand sides, each timed 3 times."""
        import numpy as np
        import torch
        p12 = self.ws.fold_rhs(self.p.view(self.N_HELD, -1))
        res = {}
        for name in ("plain", "warm"):
            ts = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                if name == "plain":
                    _, info = self.ws.solve_plain(p12, self.TOL, self.iters)
                else:
                    _, e, r, picked = self.ws.solve_warm(p12, self.TOL, self.iters)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            if name == "plain":
                infos = ss.read_infos(info, self.N_HELD)
                its = np.array([i["iters"] for i in infos])
                rho = np.array([i["rho"] for i in infos])
            else:
                its, rho = self.ws.warm_counts(ss.read_infos(e, self.N_HELD), ss.read_infos(r, self.N_HELD), self.TOL)
            res[name] = {"ms": float(np.median(ts)), "iters_mean": float(its.mean()),
                         "iters_median": float(np.median(its)), "iters_max": int(its.max()),
                         "reached": float(np.mean(rho <= self.TOL))}
        res["warm"]["kept_guess"] = float(picked.float().mean().item())
        res["warm"]["time_vs_plain_f32"] = res["warm"]["ms"] / res["plain"]["ms"]
        res["warm"]["iters_vs_plain_f32"] = res["warm"]["iters_mean"] / res["plain"]["iters_mean"]
        res["training"] = {"pairs": self.N_TRAIN, "epochs": self.EPOCHS, "seconds": self.setup_s}
        return res

    def extra(self, ss):
        import numpy as np
        import torch
        its_w, rho_w = self._counts(ss)
        p12 = self.ws.fold_rhs(self.p.view(self.N_HELD, -1))
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, info = self.ws.solve_plain(p12, self.TOL, self.iters)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        plain = ss.read_infos(info, self.N_HELD)
        its_p = np.array([i["iters"] for i in plain])
        # Launches of one warm step: fold of A (21), fold of p, 5 iterations, recombine, CNN (4 per 256 images),
        # fold of the image, two rho-only solves, pick, continuation, recombine.
        self.launches = FOLD_LAUNCHES + 1 + 1 + 1 + 4 * ((self.N_HELD + 255) // 256) + 1 + 2 + 1 + 1 + 1
        return {
            "plain": {"ms": float(np.median(ts)), "iters_mean": float(its_p.mean()),
                      "iters_median": float(np.median(its_p)), "reached": float(np.mean([i["rho"] <= self.TOL
                                                                                       for i in plain]))},
            "warm": {"iters_mean": float(its_w.mean()), "iters_median": float(np.median(its_w)),
                     "reached": float(np.mean(rho_w <= self.TOL)),
                     "fewer_iters_frac": float(np.mean(its_w < its_p))},
            "training": {"pairs": self.N_TRAIN, "epochs": self.EPOCHS, "batch": 64, "lr": 1e-3,
                         "loss_first_epoch": self.loss_hist[0], "loss_last_epoch": self.loss_hist[-1],
                         "seconds": self.setup_s},
        }

    def config(self):
        return {"workload": "learned warm start: 512 held-out phantoms on the tiny slice geometry (32x16 voxels, "
                            "M=640) reconstructed to rho <= 1e-3, lambda=1, network trained on 20000 phantoms",
                "nrhs": self.N_HELD, "N": self.g.N, "M": self.g.M, "S": self.info["S"], "tol": self.TOL,
                "max_iters": self.iters, "l2": "flushed between timed steps (256 MiB write)"}

    def oracle_case(self, budget_s):
        from oracle import geometry as ogeo
        from oracle import split as osplit
        from paper_1902_10559_gb300.synthetic import TINY, random_phantom
        A = ogeo.mirrored_system_matrix(TINY)
        A1, A2 = osplit.fold_matrix(A)
        cases = []
        for r in range(8):
            f_true = ogeo.image_to_snake(TINY, random_phantom(TINY, 5, 8, stream=10 ** 6 + r))
            p1, p2 = osplit.fold_rhs(A @ f_true)
            cases.append((1, A1, A2, p1, p2))
        return cases, "held-out phantoms"

    def oracle_run(self, osart, case):
        _, A1, A2, p1, p2 = case
        osart.split_sart(A1, A2, p1, p2, self.lam, self.iters, self.TOL)
        return 1


WORKLOADS = {"realistic": Realistic, "batch": Batch, "multi": Multi, "precision": Precision, "warmstart": Warmstart}


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
        for case in cases:
            units += wl.oracle_run(osart, case)
            done += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return units / el, {"value": units / el, "unit": wl.unit, "cores": 1, "kind": "oracle",
                        "sample": f"{done} full FP64 solves ({wl.iters}-iteration cap) from {what} (SciPy CSR, "
                                  f"single thread), {el:.1f} s; host has {os.cpu_count()} cores"}


def job_totals(step_ms, e2e_ms, solve_ms, units, steps, device):
    """Whole-job figures: the slowest rank's times and the units of all ranks.

    Returns (step_ms, e2e_ms, solve_ms, total_units), where the times are the
    maximum over ranks and total_units is the sum over ranks of units x steps.
    Without an initialised process group this is the single-process case.
    """
    import torch
    import torch.distributed as dist
    t = torch.tensor([step_ms, e2e_ms, solve_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units) * steps], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    step_ms, e2e_ms, solve_ms = t.tolist()
    return step_ms, e2e_ms, solve_ms, u.item()


def _sart_worker(args):
    """One split system's fixed-iteration solves, in a process of its own."""
    B, q, lam, iters, reps = args
    from oracle import sart as osart
    t0 = time.perf_counter()
    for _ in range(reps):
        osart.sart_fixed(B, q, lam, iters)
    return time.perf_counter() - t0


def oracle_two_process(wl, one_process_value, budget_s):
    """The paper's own scheme on the CPU (Section 2): the two split systems in two processes.

    Each process runs the same number of fixed-iteration solves of its system;
    the value counts a voxel update once both halves are done.
    """
    import multiprocessing as mp
    cases, what = wl.oracle_case(budget_s)
    n, A1, A2, p1, p2 = cases[0]
    seconds_per_solve = n * wl.iters / one_process_value  # both systems, one process
    reps = max(1, int(budget_s / seconds_per_solve))
    ctx = mp.get_context("spawn")
    with ctx.Pool(2) as pool:
        t0 = time.perf_counter()
        times = pool.map(_sart_worker, [(A1, p1, wl.lam, wl.iters, reps), (A2, p2, wl.lam, wl.iters, reps)])
        el = time.perf_counter() - t0
    units = reps * n * wl.iters
    return {"value": units / el, "unit": wl.unit, "cores": 2, "kind": "oracle, two processes",
            "sample": f"{reps} fixed {wl.iters}-iteration FP64 solves of {what} (no stop test), A1 and A2 in two "
                      f"processes (per-process {min(times):.1f}-{max(times):.1f} s, wall {el:.1f} s including process "
                      f"start)"}


def time_steps(wl, ss, steps, warmup, stream, flush, gpu_index):
    """Warm-up, then `steps` timed steps of a set-up workload, with the clocks sampled meanwhile.

    Each timed step is bracketed by CUDA events on `stream`, after an L2 flush.
    Returns (total step ms, mean solve ms, clock summary, units of one step).
    """
    import torch
    for _ in range(warmup):
        wl.step(ss, wl.p, wl.f, ss.LAYOUT_IMAGE)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    s_solve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clocks:
        for k in range(steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            wl.step(ss, wl.p, wl.f, ss.LAYOUT_IMAGE, s_solve[k])
            ends[k].record(stream)
        torch.cuda.synchronize()
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    solve_ms = sum(a.elapsed_time(b) for a, b in s_solve) / steps
    return step_ms, solve_ms, clocks.summary(), wl.units(ss)


def batch_record(ss, dev, rank, stream, flush, gpu_index, steps, warmup):
    """The 256-slice batch, timed like the main line: the HBM-bound workload of the metric."""
    import torch
    wl = Batch()
    wl.setup(ss, dev, rank)
    step_ms, solve_ms, clocks, units = time_steps(wl, ss, steps, warmup, stream, flush, gpu_index)
    rec = {"metric": wl.metric, "value": units * steps / (step_ms / 1e3), "unit": wl.unit, "steps": steps,
           "warmup": warmup, "ms_per_step": step_ms / steps, "dtype": wl.dtype, "config": wl.config(),
           "roofline": wl.roofline(ss, solve_ms), "clocks": clocks,
           "breakdown_ms": {"solve": solve_ms, "step": step_ms / steps}, "gpu_launches": wl.launches * steps}
    rec.update(wl.extra(ss, host_tracer=False))
    del wl
    torch.cuda.empty_cache()
    return rec


def solvers_time_to_tol(ss, dev, rank, tol=1e-3):
    """Iterations and time to rho <= tol of each solver against plain FP32 split-SART, one slice each.

    Noiseless projections (p = A f of a seeded phantom; with the realistic
    slice's 1% noise rho cannot reach 1e-3), FP32 systems, lambda = 1, the
    stop test every iteration. Solvers: plain SART (the library's kernel
    choice), OS-SART over folded view pairs with and without the
    non-negativity cone, and CGLS. Each is timed 3 times with CUDA events;
    the median is reported.
    """
    import numpy as np
    import torch
    from paper_1902_10559_gb300.synthetic import REALISTIC, TINY, random_phantom
    out = {}
    for name, g, cap in (("tiny", TINY, 40000), ("realistic", REALISTIC, 20000)):
        sysm = ss.fold_system(ss.make_geometry(g), ss.F32)
        img = torch.as_tensor(random_phantom(g, 6, 12, stream=1000 * rank).reshape(-1), dtype=torch.float32,
                              device=dev)
        p = torch.empty(g.M, device=dev)
        ss.project(sysm, img, p, layout=ss.LAYOUT_IMAGE)
        p12 = torch.empty(g.M // 2, 2, device=dev)
        ss.fold_rhs(sysm, p, p12)
        f12 = torch.zeros(g.N // 2, 2, device=dev)
        runs = {
            "sart": lambda o: ss.solve(sysm, p12, f12, o),
            "os_sart": lambda o: ss.solve_os(sysm, p12, f12, o),
            "os_sart_cone": lambda o: ss.solve_os(sysm, p12, f12, o, cone=True),
            "cgls": lambda o: ss.solve_cgls(sysm, p12, f12, o),
        }
        res = {}
        for form, fn in runs.items():
            opts = ss.solve_opts(cap, 1.0, tol)
            ts = []
            for _ in range(3):
                f12.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn(opts)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            info = ss.solve_result(sysm)
            res[form] = {"ms": float(np.median(ts)), "iters": info["iters"], "rho": info["rho"],
                         "reached": bool(info["rho"] <= tol)}
        for form in ("os_sart", "os_sart_cone", "cgls"):
            res[form]["time_vs_plain_f32"] = res[form]["ms"] / res["sart"]["ms"]
        res["config"] = {"M": g.M, "N": g.N, "K": g.K, "nb": g.nb, "subsets": g.K // 2 + g.K % 2,
                         "iteration_cap": cap}
        out[name] = res
        del sysm
    return out


# Example 2 (Table 1) of the paper: a direct method on an unspecified CPU, seconds. Context only.
TABLE1_PAPER_S = {32: {"full": 1.324, "split": 0.227}, 64: {"full": 73.434, "split": 3.233},
                  128: {"full": 4948.770, "split": 76.473}}


def table1_record(ss, dev, rank):
    """The direct method at the three sizes of Example 2 (Table 1), split against full, on one GPU.

    For each size: a seeded phantom, p = A f_true (consistent data, as a test
    of the solver), then
    - split: splitsart_direct_split (fold p, the normal-equation solves of A1
      and A2, Theorem 1);
    - full: splitsart_normal_solve on the full matrix (its CSR and CSC are built
      on the host by mirroring the stored half rows, Eq. 2, outside the timed
      region).
    Each is timed 3 times with CUDA events (median). The error is
    ||f - f_true|| / ||f_true||; the paper does not define its error.
    """
    import numpy as np
    import scipy.sparse as sp
    import torch
    from paper_1902_10559_gb300.synthetic import random_phantom, table1_geometries
    out = {}
    for g in table1_geometries():
        geom = ss.make_geometry(g)
        sysm = ss.fold_system(geom, ss.F64)
        f_img = torch.as_tensor(random_phantom(g, 7, 10, stream=1000 * rank), dtype=torch.float64, device=dev)
        f_true = torch.empty(g.N, dtype=torch.float64, device=dev)
        p = torch.empty(g.M, dtype=torch.float64, device=dev)
        ss.project(sysm, f_img.reshape(-1), p, layout=ss.LAYOUT_IMAGE)
        # The same image in snake order, for the error.
        f12 = torch.empty(g.N // 2, 2, dtype=torch.float64, device=dev)
        ss.fold_image(sysm, f_img.reshape(-1), f12, layout=ss.LAYOUT_IMAGE)
        ss.recombine(sysm, f12, f_true)
        rp, col, val = ss.full_csr(geom)
        A = sp.csr_matrix((val, col, rp), shape=(g.M, g.N))
        A.sort_indices()
        T = sp.csc_matrix(A)
        T.sort_indices()
        to = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x).astype(dt), device=dev)
        csr = (to(A.indptr, np.int32), to(A.indices, np.int32), to(A.data, np.float64))
        csc = (to(T.indptr, np.int32), to(T.indices, np.int32), to(T.data, np.float64))
        res = {}
        for mode in ("split", "full"):
            solver = ss.DenseSolver(g.N // 2 if mode == "split" else g.N, device=dev)
            f = torch.zeros(g.N, dtype=torch.float64, device=dev)
            ts = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                if mode == "split":
                    ss.direct_split(sysm, solver, p, f)
                else:
                    ss.normal_solve(solver, g.M, g.N, csr, csc, p, f)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            err = float(((f - f_true).norm() / f_true.norm()).item())
            res[mode] = {"ms": float(np.median(ts)), "status": solver.result(), "error_vs_f_true": err}
            del solver
            torch.cuda.empty_cache()
        res["full_over_split"] = res["full"]["ms"] / res["split"]["ms"]
        res["size"] = {"voxels": f"{g.nx}x{g.nz}", "positions": g.K, "bins": g.nb, "M": g.M, "N": g.N}
        res["paper_cpu_s"] = TABLE1_PAPER_S[g.nx]
        out[f"{g.nx}x{g.nz}"] = res
    out["note"] = ("FP64 normal equations (B = A^T A, blocked Cholesky, two triangular solves) on the GPU; the paper's "
                   "seconds are a direct method on an unspecified CPU, context only")
    return out


def time_to_tol_record(ss, dev, rank, stream):
    """Iterations and time to rho <= 1e-3 of each form against plain FP32 split-SART, on one GPU.

    - Storage forms: FP32, BF16 and FP16 matrix values on 64 right-hand sides
      (tiny slice geometry, lambda = 1), one solve_multi launch each.
    - Learned warm start against plain FP32 from zero on 512 held-out
      right-hand sides: the whole warm pipeline (5 iterations, network, fold,
      fallback, continuation) against the plain solve.
    """
    import torch
    pr = Precision()
    pr.setup(ss, dev, rank)
    forms = pr.time_to_tol(ss)
    del pr
    ws = Warmstart()
    ws.setup(ss, dev, rank)
    warm = ws.time_to_tol(ss)
    del ws
    torch.cuda.empty_cache()
    solvers = solvers_time_to_tol(ss, dev, rank)
    return {"tol": 1e-3, "forms_64rhs": forms, "warm_start_512rhs": warm, "solvers_one_slice": solvers,
            "note": "ms = launch (or pipeline) time until the last right-hand side stops, median of 3; "
                    "time_vs_plain_f32 < 1 is a gain"}


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

    if ws > 1:
        dist.barrier()
    step_ms, solve_ms, clocks, units = time_steps(wl, ss, args.steps, args.warmup, stream, flush, local)
    if ws > 1:
        dist.barrier()

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

    step_ms, e2e_ms, solve_ms, total_units = job_totals(step_ms, e2e_ms, solve_ms, units, args.steps, dev)
    value = total_units / (step_ms / 1e3)
    e2e_value = total_units / (e2e_ms / 1e3)
    extra = wl.extra(ss)
    out = {
        "metric": wl.metric, "value": value, "unit": wl.unit, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": wl.higher_is_better,
        "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype,
        "data": "synthetic (seeded random ellipses, Siddon projections)",
        "config": wl.config(),
        "e2e": {"value": e2e_value, "unit": wl.unit, "h2d_bytes_per_step": wl.p.numel() * 4,
                "d2h_bytes_per_step": wl.f.numel() * 4,
                "path": "the Python binding over the C ABI; the host<->device copies are torch's pinned-memory "
                        "copies, outside the library (its entry points take device pointers)"},
        "gpu_launches": wl.launches * args.steps,
        "roofline": wl.roofline(ss, solve_ms),
        "clocks": clocks,
        "breakdown_ms": {"solve": solve_ms, "fold_A": fold_ms, "step": step_ms / args.steps},
    }
    out.update(extra)
    if args.workload == "realistic" and not args.no_extras:
        # The metric's other two clauses, on the same GPU in the same run: the HBM roofline
        # on the batch (whose inputs far exceed L2) and the time to rho <= 1e-3 of each form.
        del wl
        torch.cuda.empty_cache()
        out["batch"] = batch_record(ss, dev, rank, stream, flush, local, args.batch_steps, 3)
        out["time_to_tol"] = time_to_tol_record(ss, dev, rank, stream)
        out["table1_direct"] = table1_record(ss, dev, rank)
    if rank == 0 and not args.no_cpu_baseline:
        wl0 = WORKLOADS[args.workload]()
        _, out["cpu_baseline"] = oracle_throughput(wl0, args.cpu_seconds)
        if wl0.two_process_baseline:
            out["cpu_baseline_2proc"] = oracle_two_process(wl0, out["cpu_baseline"]["value"], args.cpu_seconds)
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
        osart.split_sart(A1, A2, p1, p2, wl.lam, 5)  # short warm-up solves
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        for case in cases:
            units += wl.oracle_run(osart, case)
    total = time.perf_counter() - t0
    value = units / total
    cfg = {"workload": f"oracle on {what} of the {args.workload} workload", "iterations": wl.iters,
           "lambda": wl.lam}
    out = {"impl": "reference", "metric": wl.metric, "value": value, "unit": wl.unit, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": wl.higher_is_better, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": wl.unit, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} x {what}, full solves ({wl.iters}-iteration cap; SciPy CSR, "
                                      f"single thread); host has {os.cpu_count()} cores"},
           "e2e": {"value": value, "unit": wl.unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps; default: the workload's, long enough (about 0.2 s or more) for the clock "
                         "sampler to see the GPU under load; 3 for the reference arm")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="realistic")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--slices", type=int, default=256, help="batch workload: number of slices (first n of the 256)")
    ap.add_argument("--no-extras", action="store_true",
                    help="realistic workload: skip the batch record and the time-to-tolerance record")
    ap.add_argument("--batch-steps", type=int, default=5, help="timed steps of the batch record")
    args = ap.parse_args()
    Batch.n_slices = max(1, min(256, args.slices))
    if args.steps is None:
        args.steps = 3 if args.impl == "reference" else WORKLOADS[args.workload].default_steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
