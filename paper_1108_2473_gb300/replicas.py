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


_HOST_GROUP = {}


def host_group(force_new: bool = False):
    """A process group that reduces CPU tensors: the default group when its
    backend is gloo, otherwise (NCCL, as bench.py creates under torchrun) a gloo
    group over the same ranks, created once.  Every rank must call this
    together the first time (group creation is collective)."""
    if not force_new and dist.get_backend() == "gloo":
        return None
    key = "forced" if force_new else "gloo"
    if key not in _HOST_GROUP:
        _HOST_GROUP[key] = dist.new_group(backend="gloo")
    return _HOST_GROUP[key]


def combine_loops(per_t: torch.Tensor, n_vectors_here: int, device=None, group=None):
    """Average per-time-slice loop sums over all ranks' noise vectors.

    per_t holds this rank's sum over its vectors; returns (total / n_total) on
    every rank.  The reduction runs on a CPU-side copy through a gloo group
    (host_group()), so no GPU collective is involved whatever backend the
    default process group uses.
    """
    local = torch.view_as_real(per_t.detach().to("cpu", torch.complex128)).clone()
    n = torch.tensor([float(n_vectors_here)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        g = group if group is not None else host_group()
        dist.all_reduce(local, op=dist.ReduceOp.SUM, group=g)
        dist.all_reduce(n, op=dist.ReduceOp.SUM, group=g)
    return torch.view_as_complex(local) / n.item()
