"""Multi-GPU execution by independent replicas (one process per GPU).

Ciphertexts are independent, so ranks never exchange ring data: each rank
holds its own keys and processes its own ciphertexts, and the only
collectives are the host-side barrier and the reduction of the timing
(maximum over ranks) and of the work done (sum over ranks).
"""
from __future__ import annotations


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s keys and inputs: distinct per rank, reproducible."""
    return int(base) * 1000003 + int(rank)


def aggregate(units: float, seconds: float, dist=None):
    """(whole-job units per second, max seconds over ranks, total units) for this rank's
    `units` processed in `seconds`; without an initialised process group, the local values."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return units / seconds, seconds, units
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())
