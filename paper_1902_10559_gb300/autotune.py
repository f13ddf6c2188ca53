"""Autotuner for the split-SART launch shapes.

Each tunable is timed with a short solve and the fastest is kept. Choices are
cached per (device, storage type, problem class) in a JSON file:
$SPLITSART_TUNE_CACHE, or ~/.cache/splitsart/tune.json.

- Persistent solve: kernel (shared-memory resident, tile streaming, row
  streaming through registers, row streaming in compacted index order fed
  per warp or through a producer warp's shared-memory ring, or per-warp
  bulk-staged streaming), tile entries per CTA (chunk entries of the ring),
  lanes per column in the back-projection, threads per CTA.
- Multi-right-hand-side solve: right-hand sides per CTA, threads per CTA,
  lanes per row and right-hand side.

The tuner only chooses among launch shapes of the same arithmetic, so every
choice gives a result within rounding of every other.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import threading

from . import splitsart as ss

_LOCK = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("SPLITSART_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "splitsart", "tune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # the cache is an optimisation only


def problem_class(system: ss.System) -> str:
    """Device, storage type, batch-ness and log2 size bins of S, Mh and Nh."""
    import torch
    info = system.info()
    b = lambda x: int(math.log2(max(int(x), 1)))
    dev = torch.cuda.get_device_name()
    return f"{dev}|dt{system.dtype}|ns{'1' if system.nslices == 1 else 'n'}|S{b(info['S'])}|M{b(info['Mh'])}|N{b(info['Nh'])}"


def _time_solve(system, p12, f12, opts, reps: int = 3) -> float:
    import torch
    f0 = f12.clone()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for r in range(reps + 1):
        f12.copy_(f0)
        ev0.record()
        ss.solve(system, p12, f12, opts)
        ev1.record()
        torch.cuda.synchronize()
        if r:
            best = min(best, ev0.elapsed_time(ev1))
    f12.copy_(f0)
    return best


def solve_candidates(system: ss.System) -> list[dict]:
    out = []
    if system.nslices == 1:
        for lpc in (4, 8, 16):
            for bt in (256, 384, 512):
                for rw in (0, 160, 320):  # rows' fixed weight in the CTA row plan (0 = library default)
                    out.append({"kernel": 2, "lanes_per_col": lpc, "block_threads": bt, "tile_entries": 0,
                                "row_weight": rw})
    for kern, bts in ((4, (256, 384)), (3, (256, 512)), (5, (256, 512))):
        for lpc in ((4, 8) if kern in (4, 5) else (4, 8, 16)):
            for bt in bts:
                out.append({"kernel": kern, "lanes_per_col": lpc, "block_threads": bt, "tile_entries": 0})
    for lpc in (4, 8):  # kernel 7 ignores block_threads; tile_entries is its chunk entry target
        for te in (0, 2048, 6144):
            out.append({"kernel": 7, "lanes_per_col": lpc, "block_threads": 0, "tile_entries": te})
    for lpc in (4, 8, 16):
        for te in (4096, 8192, 12288):
            if system.dtype == ss.F64 and te > 8192:
                continue
            for bt in (512, 1024):
                out.append({"kernel": 1, "lanes_per_col": lpc, "block_threads": bt, "tile_entries": te})
    return out


def tune_solve(system: ss.System, p12, f12, iters: int = 10, use_cache: bool = True) -> dict:
    """Return the fastest launch shape for ``system``, as solve_opts keyword arguments.

    p12 and f12 are real inputs of the right size. f12 is restored after the
    timing runs.
    """
    key = "solve|" + problem_class(system)
    with _LOCK:
        cache = _load() if use_cache else {}
        if key in cache:
            return dict(cache[key])
        best, best_t = None, float("inf")
        for c in solve_candidates(system):
            try:
                t = _time_solve(system, p12, f12, ss.solve_opts(iters, 1.0, **c))
            except ss.SplitSartError:
                continue  # a shape this system cannot use (shared memory, sizes)
            if t < best_t:
                best, best_t = c, t
        if best is None:
            best = {"kernel": 0, "lanes_per_col": 0, "block_threads": 0, "tile_entries": 0}
        if use_cache:
            cache[key] = best
            _store(cache)
        return dict(best)


def tune_multi(system: ss.System, p12, f12, iters: int = 10, use_cache: bool = True) -> dict:
    """Return the fastest (rhs_per_cta, block_threads, lanes_per_row) for solve_multi on this system and
    right-hand-side count (lanes_per_row: lanes per row and right-hand side, 2, 4 or 8)."""
    import torch
    nrhs = p12.shape[0]
    key = f"multi|{nrhs}|" + problem_class(system)
    with _LOCK:
        cache = _load() if use_cache else {}
        if key in cache:
            return dict(cache[key])
        info = torch.zeros(nrhs * ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device="cuda")
        f0 = f12.clone()
        best, best_t = None, float("inf")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rc in (1, 2, 4, 8, 16):
            for bt in (128, 256, 512, 640, 768, 1024):
                for lpr in (2, 4, 8):
                    if rc * lpr > 32:
                        continue
                    try:
                        ts = []
                        for r in range(3):
                            f12.copy_(f0)
                            ev0.record()
                            ss.solve_multi(system, p12, f12,
                                           ss.solve_opts(iters, 1.0, block_threads=bt, lanes_per_row=lpr), info,
                                           rhs_per_cta=rc)
                            ev1.record()
                            torch.cuda.synchronize()
                            ts.append(ev0.elapsed_time(ev1))
                    except ss.SplitSartError:
                        continue
                    t = min(ts[1:])
                    if t < best_t:
                        best, best_t = {"rhs_per_cta": rc, "block_threads": bt, "lanes_per_row": lpr}, t
        f12.copy_(f0)
        if best is None:
            best = {"rhs_per_cta": 0, "block_threads": 0, "lanes_per_row": 0}
        if use_cache:
            cache[key] = best
            _store(cache)
        return dict(best)
