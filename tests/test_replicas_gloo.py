"""World-size-2 gloo tests (CPU) of the replica host logic: disjoint noise
vectors per rank, the max-over-ranks timing, and the combination of the
ranks' per-time-slice loops, which must equal a single process's estimate."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1108_2473_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _per_t_of(index, lt=4):
    # deterministic stand-in for one noise vector's per-time-slice loops
    rng = np.random.default_rng(1000 + index)
    return rng.standard_normal((lt, 6)) + 1j * rng.standard_normal((lt, 6))


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        idx = replicas.noise_indices(rank, world, 3)
        acc = sum(_per_t_of(i) for i in idx)
        comb = replicas.combine_loops(torch.from_numpy(acc), len(idx))
        # the path taken under an NCCL default group: a separate gloo group
        comb2 = replicas.combine_loops(torch.from_numpy(acc), len(idx), group=replicas.host_group(force_new=True))
        tmax = replicas.max_over_ranks(1.0 + rank)
        out.put((rank, idx, comb.numpy(), tmax, comb2.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_combine():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    all_idx = res[0][1] + res[1][1]
    assert len(set(all_idx)) == len(all_idx) == 6  # disjoint
    expect = sum(_per_t_of(i) for i in all_idx) / 6
    for r in res:
        assert np.allclose(r[2], expect, atol=1e-14, rtol=0)
        assert np.array_equal(r[4], r[2])
        assert r[3] == 2.0  # max over ranks


def test_single_process_is_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    x = torch.ones((4, 6), dtype=torch.complex128) * 2
    assert torch.allclose(replicas.combine_loops(x, 2), x / 2)
    assert replicas.noise_indices(1, 4, 2, first=10) == [11, 15]
    with pytest.raises(ValueError):
        replicas.noise_indices(4, 4, 1)
