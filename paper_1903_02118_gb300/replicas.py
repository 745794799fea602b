"""Process-group plumbing for runs on several GPUs of one node (one process per GPU).

The FDP=H step of one scenario is not split across GPUs here: N GPUs run N independent replicas
(separate scenarios, weak scaling), so the data path has no collective.  What the ranks share is
the timing protocol: a barrier before and after the timed region and the maximum of the ranks'
elapsed times.  With the NCCL backend the reduction goes through a device tensor, with gloo
(CPU tests) through a host tensor.
"""
import os


def init():
    """(world, rank, local_rank) from the launcher's environment; joins the process group when
    world > 1 (NCCL if CUDA is available, else gloo)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def _device():
    import torch
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world):
    """Largest `value` over the ranks (every rank gets it)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world):
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
