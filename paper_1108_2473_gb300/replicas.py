"""Replica sharding for several GPUs (one process per GPU).

The loop estimator is a sum over independent noise vectors (Eq. loop
stochastic), so ranks share no data while they work: rank r of N takes the
noise vectors r, r + N, r + 2N, ...  The only exchanges are on the host side
of a job: the maximum of the ranks' timings, and the sum of the ranks'
per-time-slice loop arrays ([Lt][6] complex, a few KB) at the end.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def noise_indices(rank: int, world: int, count: int, first: int = 0):
    """Noise-vector indices of this rank: `count` of them, disjoint across ranks."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return [first + rank + world * k for k in range(count)]


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the job's wall time); identity without a process group."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_loops(per_t: torch.Tensor, n_vectors_here: int, device=None):
    """Average per-time-slice loop sums over all ranks' noise vectors.

    per_t holds this rank's sum over its vectors; returns (total / n_total) on
    every rank.  The reduction is done on a CPU-side copy, so no GPU
    collective is involved.
    """
    local = torch.view_as_real(per_t.detach().to("cpu", torch.complex128)).clone()
    n = torch.tensor([float(n_vectors_here)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(local, op=dist.ReduceOp.SUM)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return torch.view_as_complex(local) / n.item()
