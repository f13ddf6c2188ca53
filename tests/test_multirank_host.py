"""Host-side logic of the multi-rank bench path, on two gloo ranks (CPU).

Each rank reconstructs its own slices (no data-path collective). The job's
figures are the slowest rank's times and the sum of all ranks' units.
"""
import multiprocessing as mp
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_totals_take_max_time_and_sum_units():
    from tests.multirank_worker import totals_worker
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=totals_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        step_ms, e2e_ms, solve_ms, units = results[r]
        assert (step_ms, e2e_ms, solve_ms) == (11.0, 22.0, 6.0)
        assert units == (100 + 200) * 3


def test_single_process_totals():
    import torch

    import bench
    assert bench.job_totals(4.0, 5.0, 3.0, 7, 2, torch.device("cpu")) == (4.0, 5.0, 3.0, 14.0)


def test_ranks_draw_different_phantoms():
    """Rank r's slices use seed streams 1000 r + 2 k, so ranks never duplicate work."""
    from paper_1902_10559_gb300.synthetic import TINY, random_phantom
    a = random_phantom(TINY, 2, 20, stream=1000 * 0)
    b = random_phantom(TINY, 2, 20, stream=1000 * 1)
    assert not np.array_equal(a, b)
