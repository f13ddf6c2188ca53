"""Host-side checks of the launch-shape autotuner (no GPU).

- The candidate lists hold only shapes the C ABI accepts, and the resident
  kernel only for single-slice systems.
- The problem class separates storage types, batches and size bins.
- The cache round-trips through its JSON file: a second tune call returns
  the stored choice without timing anything.
"""
import json
import types

import pytest

from paper_1902_10559_gb300 import autotune
from paper_1902_10559_gb300 import splitsart as ss


class FakeSystem:
    """The attributes the tuner reads from a splitsart.System."""

    def __init__(self, dtype=ss.F32, nslices=1, S=1_400_088, Mh=13312, Nh=32768):
        self.dtype = dtype
        self.nslices = nslices
        self._info = {"S": S, "Mh": Mh, "Nh": Nh}

    def info(self):
        return dict(self._info)


@pytest.fixture
def fake_device(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "NVIDIA GB300")


@pytest.fixture
def cache_file(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SPLITSART_TUNE_CACHE", str(path))
    return path


VALID_LPC = {1, 2, 4, 8, 16, 32}


@pytest.mark.parametrize("dtype", [ss.F64, ss.F32, ss.BF16])
@pytest.mark.parametrize("nslices", [1, 3])
def test_candidates_are_valid_launch_shapes(dtype, nslices):
    cands = autotune.solve_candidates(FakeSystem(dtype, nslices))
    assert cands
    keys = {"kernel", "lanes_per_col", "block_threads", "tile_entries"}
    seen = set()
    for c in cands:
        assert keys <= set(c)
        seen.add(tuple(sorted(c.items())))
        assert c["kernel"] in (1, 2, 3, 4, 5, 7)  # never 6 or 8: the implicit fold changes the rounding
        assert c["lanes_per_col"] in VALID_LPC
        bt = c["block_threads"]
        if c["kernel"] == 7:  # a fixed CTA shape (producer warp + consumers); tile_entries = chunk target
            assert bt == 0 and c["lanes_per_col"] in (4, 8)
            te = c["tile_entries"]
            assert te == 0 or (te % 1024 == 0 and 1024 <= te <= 16384)
            ss.solve_opts(10, 1.0, **c)
            continue
        assert bt % 32 == 0 and 64 <= bt <= 1024
        if c["kernel"] in (2, 3, 5):
            assert bt <= 512
        if c["kernel"] == 5:
            assert c["lanes_per_col"] in (4, 8)
        if c["kernel"] == 4:
            assert bt <= 384 and c["lanes_per_col"] in (4, 8)
        if c["kernel"] == 1:
            te = c["tile_entries"]
            assert te % 1024 == 0 and 1024 <= te <= 16384
            if dtype == ss.F64:
                assert te <= 8192  # FP64 pairs are twice as wide
        else:
            assert c["tile_entries"] == 0
        if c["kernel"] == 2:
            assert nslices == 1  # the resident kernel has no per-slice stop tests
        # All fields are plain keyword arguments of solve_opts.
        ss.solve_opts(10, 1.0, **c)
    assert len(seen) == len(cands)  # no candidate is timed twice


def test_problem_class_separates_types_batches_and_sizes(fake_device):
    base = autotune.problem_class(FakeSystem())
    assert base.startswith("NVIDIA GB300|")
    assert autotune.problem_class(FakeSystem(dtype=ss.BF16)) != base
    assert autotune.problem_class(FakeSystem(nslices=4)) != base
    assert autotune.problem_class(FakeSystem(S=4 * 1_400_088)) != base
    # Sizes within one power of two share a class (log2 bins).
    assert autotune.problem_class(FakeSystem(S=1_500_000, Mh=14000, Nh=40000)) == base


def test_cache_round_trip(cache_file, fake_device, monkeypatch):
    sysm = FakeSystem()
    timed = []

    def fake_time(system, p12, f12, opts, reps=3):
        timed.append((opts.kernel, opts.lanes_per_col, opts.block_threads, opts.tile_entries, opts.row_weight))
        # The row-streaming kernel with 8 lanes per column and 512 threads is "fastest".
        return 1.0 if (opts.kernel, opts.lanes_per_col, opts.block_threads) == (3, 8, 512) else 2.0

    monkeypatch.setattr(autotune, "_time_solve", fake_time)
    first = autotune.tune_solve(sysm, None, None)
    assert (first["kernel"], first["lanes_per_col"], first["block_threads"]) == (3, 8, 512)
    assert len(timed) == len(autotune.solve_candidates(sysm))
    stored = json.loads(cache_file.read_text())
    assert stored["solve|" + autotune.problem_class(sysm)] == first

    def no_timing(*a, **k):
        raise AssertionError("a cached class must not be timed again")

    monkeypatch.setattr(autotune, "_time_solve", no_timing)
    assert autotune.tune_solve(sysm, None, None) == first
    # Without the cache the tuner times again.
    monkeypatch.setattr(autotune, "_time_solve", fake_time)
    timed.clear()
    assert autotune.tune_solve(sysm, None, None, use_cache=False) == first and timed


def test_rejected_shapes_are_skipped(cache_file, fake_device, monkeypatch):
    """A shape the library refuses (too much shared memory, say) is skipped, not fatal."""
    def refuse_resident(system, p12, f12, opts, reps=3):
        if opts.kernel == 2:
            raise ss.SplitSartError(ss.ERR_ARG, "does not fit")
        return 5.0 - 0.001 * opts.block_threads

    monkeypatch.setattr(autotune, "_time_solve", refuse_resident)
    best = autotune.tune_solve(FakeSystem(), None, None)
    assert best["kernel"] != 2


def test_unreadable_cache_is_ignored(cache_file, fake_device, monkeypatch):
    cache_file.write_text("{not json")
    monkeypatch.setattr(autotune, "_time_solve", lambda *a, **k: 1.0)
    best = autotune.tune_solve(FakeSystem(), None, None)
    assert best == json.loads(cache_file.read_text())["solve|" + autotune.problem_class(FakeSystem())]
