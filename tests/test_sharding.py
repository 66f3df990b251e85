"""Chain sharding across ranks, on CPU: shard ranges, and a world-size-2
gloo run whose ranks each sweep their shard (FP64 oracle, global chain
indices) and sum their counts with the sharding helper; the total must equal
the counts of one unsharded run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_18456_gb300 import sharding, synth


@pytest.mark.parametrize("M,world", [(10, 2), (11, 2), (7, 3), (1, 1), (5, 8), (10000, 4)])
def test_shard_range_partitions(M, world):
    spans = [sharding.shard_range(M, r, world) for r in range(world)]
    covered = [k for first, n in spans for k in range(first, first + n)]
    assert covered == list(range(M))
    sizes = [n for _, n in spans]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_shard_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        sharding.shard_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, M, L, q, seed, nsweeps):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc  # test infrastructure: the FP64 reference of each shard's work
        h, J = synth.planted_local_model(L, q, 5, sigma_h=1.0, sigma_J=0.3)
        h64, J64 = h.astype(np.float64), J.astype(np.float64)
        first, n = sharding.shard_range(M, rank, world)
        S = orc.chains_init(n, L, q, seed, first)
        S = orc.gibbs(h64, J64, S, seed, 0, nsweeps, 1.0, first)
        counts = torch.from_numpy(orc.chain_stats(S, q).astype(np.int32))
        sharding.allreduce_counts(counts)
        full = orc.gibbs(h64, J64, orc.chains_init(M, L, q, seed, 0), seed, 0, nsweeps, 1.0, 0)
        ref = orc.chain_stats(full, q)
        assert np.array_equal(counts.numpy(), ref), f"rank {rank}: summed shard counts differ"
        # every rank holds the same totals
        tot = torch.tensor([int(counts.sum())], dtype=torch.int64)
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        assert int(tot) == int(counts.sum())
    finally:
        dist.destroy_process_group()


def test_sharded_counts_equal_unsharded_gloo(orc):
    mp.start_processes(_rank_main, args=(2, _free_port(), 37, 9, 5, 77, 3), nprocs=2, join=True,
                       start_method="spawn")
