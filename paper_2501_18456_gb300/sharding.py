"""Chain sharding across ranks (one process per GPU).

The M chains of a run are independent (Sec. 2.1), so they split into
contiguous shards, one per rank, with h and J replicated.  Every draw is
keyed by the GLOBAL chain index (bm_chains_init_shard), so the shards draw
exactly the states of one unsharded run.  The only exchange is the sum of
the int32 pair counts before the update (exact); every rank then applies the
same deterministic bm_update with the total chain count, so the replicas'
parameters stay identical.

bench.py --gpus N runs N independent replicas (weak scaling, no collective
on the data path); these helpers give the sharded alternative, with the one
all-reduce above, and are exercised by world-size-2 gloo runs on CPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(M: int, rank: int, world: int) -> tuple[int, int]:
    """(first global chain, number of chains) of `rank`'s shard: contiguous,
    sizes differing by at most one, the larger shards first."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    base, extra = divmod(M, world)
    n = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, n


def allreduce_counts(counts: torch.Tensor, group=None) -> torch.Tensor:
    """Sums the int32 pair counts of all ranks in place (exact)."""
    if counts.dtype != torch.int32:
        raise TypeError("pair counts are int32")
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts


def sharded_step(bm, model, chains, counts, fi, fij, M_total: int, nsweeps: int, lr: float,
                 target: float, group=None, stream=None):
    """One training iteration of a shard: sweeps of the local chains, local
    counts, global counts, identical update on every rank.  Returns
    (pearson, applied) as bm_update does."""
    bm.bm_gibbs_sweep(model, chains, nsweeps, 1.0, stream)
    bm.bm_chain_stats(chains, counts, stream)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        if counts.is_cuda:
            torch.cuda.synchronize()  # the counts were written on the library's stream
        allreduce_counts(counts, group)
    return bm.bm_update(model, fi, fij, counts, M_total, lr, target, True, stream)
