"""Multi-GPU runs as independent replicas (one process per GPU).

The tiled QR of one matrix runs on one GPU here; N GPUs run N independent problems,
each rank its own seeded input, and a batch of independent matrices is split across
ranks by matrix index.  The only cross-rank operations are barriers around a timed
region and the maximum over ranks of the measured times - no data moves between GPUs.
Launched by torchrun (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* in the environment);
NCCL on GPUs, gloo on CPU (tests).
"""
from __future__ import annotations

import os


def env_ranks():
    """(rank, local_rank, world_size) from the launcher's environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def init(backend: str = "nccl", device=None) -> None:
    """Joins the process group when more than one rank runs."""
    import torch.distributed as dist
    _, _, world = env_ranks()
    if world > 1 and not dist.is_initialized():
        if device is not None and backend == "nccl":
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity for 1 rank)."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank's independent problem (rank 0 keeps the single-GPU seed)."""
    return base + 1000 * rank


def shard(count: int, rank: int, world: int):
    """Indices of a batch of ``count`` items that rank processes: every world-th item,
    so that the ragged size mix is spread evenly."""
    return list(range(rank, count, world))


def finalize() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()
