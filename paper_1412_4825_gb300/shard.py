"""Chain sharding across ranks (one process per GPU).

Chains (and streams) are independent units: the global chain id is part of
every Philox counter the chain uses, so a chain gives the same bits whichever
rank runs it and however the range is cut.  Sharding therefore needs no
exchange while sweeping; the only collective steps are a final gather of
per-chain state and moments in rank order (deterministic concatenation, no
floating-point reduction) and the maximum of the ranks' timings.

The full LDA step is the exception with a real exchange: its documents are
sharded the same way, but the word-topic and topic counts are shared by the
whole corpus, so after every sweep each rank's count changes are summed over
the ranks (`lda_exchange`, an integer all-reduce: exact and independent of the
order of the additions) before they are added into every rank's copy.

Two partitions:
  * `chain_range`: a fixed total split into contiguous, balanced ranges
    (strong scaling);
  * `weak_range`: every rank takes the same count, rank r the r-th block of
    global ids (weak scaling; the total grows with the ranks).
"""
from __future__ import annotations


def chain_range(n_total: int, world: int, rank: int):
    """(chain_offset, n_chains) of `rank` when `n_total` chains are split over
    `world` ranks: contiguous, sizes differing by at most one, lower ranks
    taking the remainder."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad partition: n_total=%d world=%d rank=%d" % (n_total, world, rank))
    base, rem = divmod(n_total, world)
    offset = rank * base + min(rank, rem)
    return offset, base + (1 if rank < rem else 0)


def weak_range(per_rank: int, rank: int):
    """(chain_offset, n_chains) of `rank` when each rank runs `per_rank` chains."""
    if per_rank < 0 or rank < 0:
        raise ValueError("bad partition: per_rank=%d rank=%d" % (per_rank, rank))
    return rank * per_rank, per_rank


def gather_rows(dist, local, n_total: int, world: int, rank: int, dst: int = 0):
    """Concatenate each rank's rows (a tensor whose first dimension is its
    chain range from `chain_range(n_total, world, r)`) in rank order on rank
    `dst`; other ranks get None.  Rows are padded to the largest range, so
    one all_gather of equal shapes serves any backend."""
    import torch

    counts = [chain_range(n_total, world, r)[1] for r in range(world)]
    if local.shape[0] != counts[rank]:
        raise ValueError("rank %d holds %d rows, its range has %d" % (rank, local.shape[0], counts[rank]))
    width = max(counts)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    if rank != dst:
        return None
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def max_over_ranks(dist, value: float, device="cpu") -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def lda_exchange(dist, dnkw):
    """Sum the ranks' count changes of one sweep of the full LDA step in place
    (int32 [V*K + K] on the ranks' devices or hosts: word-topic, then topic)."""
    dist.all_reduce(dnkw, op=dist.ReduceOp.SUM)
    return dnkw
