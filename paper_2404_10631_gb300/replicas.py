"""Multi-GPU form of the classification path: replicas.

Frames are independent (the paper classifies each captured cube on its own),
so N GPUs run N copies of the path, one process per GPU, each on its own
frames, with no exchange on the data path. The process group only lines the
ranks up around a timed region and takes the slowest rank's time, so that a
whole-job rate counts every rank's frames over the time the last one needed.

The helpers below are that host logic. They run unchanged under NCCL (one
GPU per rank, the tensors on the rank's device) and under gloo (CPU ranks),
which is how they are tested without GPUs.
"""

import os


def env_ranks():
    """(world_size, rank, local_rank) from the launcher's environment
    (torchrun sets WORLD_SIZE, RANK, LOCAL_RANK; a plain run is one rank)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world, local=0, backend="nccl"):
    """Join the process group when world > 1: NCCL bound to GPU `local`, or
    `backend` ("gloo") for CPU ranks. MASTER_ADDR / MASTER_PORT come from the
    environment (127.0.0.1 on a single node)."""
    if world <= 1:
        return
    import torch
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)


def barrier(world):
    """Every rank reaches this point before any goes on (no-op for one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of `values` (floats) over the ranks: the slowest
    rank's time for each timed region. `device`: where the reduction tensor
    lives (the rank's GPU under NCCL, None = CPU for gloo)."""
    vals = [float(v) for v in values]
    if world <= 1:
        return vals
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu().tolist()]


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units per second of the whole job: every rank processed
    `units_per_rank` (weak scaling: the same work per rank), the job took the
    slowest rank's `seconds_max`."""
    if seconds_max <= 0.0:
        raise ValueError("seconds_max must be positive")
    return world * float(units_per_rank) / float(seconds_max)


def reports(rank):
    """Only rank 0 prints the job's result line."""
    return rank == 0


def finalize(world):
    """Leave the process group (no-op for one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
