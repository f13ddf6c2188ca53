"""Worker of the two-rank host tests (spawned processes, gloo on CPU)."""
import os


def totals_worker(rank, world_size, port, queue):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        import torch

        import bench
        out = bench.job_totals(10.0 + rank, 20.0 + 2 * rank, 5.0 + rank, 100 * (rank + 1), 3, torch.device("cpu"))
        queue.put((rank, out))
    finally:
        dist.destroy_process_group()
