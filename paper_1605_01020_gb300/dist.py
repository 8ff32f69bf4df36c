"""Multi-process bookkeeping for the element-local path.

The element-local problem has no exchange step when every rank condenses its own
mesh, so the multi-GPU mode is weak scaling: each rank runs the same-sized
workload, the job time is the maximum over ranks and the job throughput counts the
elements of all ranks.  Works with any torch.distributed backend (nccl on GPUs,
gloo on CPU for tests)."""
import torch


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity if the
    process group is not initialised)."""
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def weak_scaling_throughput(units_per_rank, steps, ms_local, device=None):
    """(units/s of the whole job, max-over-ranks milliseconds)."""
    world = torch.distributed.get_world_size() if (torch.distributed.is_available()
                                                   and torch.distributed.is_initialized()) else 1
    (ms,) = max_over_ranks([ms_local], device)
    return units_per_rank * steps * world / (ms / 1e3), ms
