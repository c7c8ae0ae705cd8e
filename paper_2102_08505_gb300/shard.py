"""Host-side logic for runs on several GPUs of one node (one process per GPU).

Single-matrix SP2 is run as independent replicas (each rank its own Hamiltonian), and
batched SP2 deals whole matrices to ranks; neither needs a collective on the data path.
The only collectives are a barrier around the timed region and a maximum over ranks
of the elapsed time.
"""
import os


def rank_info():
    """(rank, local_rank, world_size) from the launcher's environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def deal(work, world):
    """Longest-processing-time assignment of items with the given work estimates to
    `world` ranks: items in decreasing work (ties by index) go to the least-loaded rank
    (ties by rank).  Deterministic, so every rank computes the same split.  Returns a
    list of sorted index lists, one per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(work[i])
    return [sorted(p) for p in parts]


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks of the default process group (the value itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    """Sum of a float over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
