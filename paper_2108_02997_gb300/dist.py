"""Multi-GPU plumbing for runs with one process per GPU (torchrun).

PageRank instances are independent (Sections 2-4 solve each (graph, alpha,
tau, norm) on its own), so a multi-GPU run gives every rank its own batch of
instances and no data-path collective exists: ranks meet only at barriers
around a timed region and in one max-reduction of its duration. The helpers
take the backend from the device: NCCL for CUDA ranks, gloo for CPU ranks
(how the host logic is tested without GPUs).
"""
import os


def env():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(device="cuda"):
    """Join the process group when WORLD_SIZE > 1; returns (world, rank, local)."""
    world, rank, local = env()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if device == "cuda" else "gloo")
    return world, rank, local


def finish(world):
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


def barrier(world, device="cuda"):
    """Every rank arrives; with CUDA, also every queued kernel of this rank ends."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if device == "cuda":
        import torch
        torch.cuda.synchronize()


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest of the ranks' values of x (x itself alone)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s copy of a workload: rank 0 keeps the workload's
    own seed, others draw graphs of the same shape from disjoint seeds."""
    return seed if rank == 0 else seed + 1_000_003 * rank
