"""Chain sharding across processes (one GPU per process) and the host-side reduction.

Chains are independent Markov chains ("one Markov chain for each configuration",
Algorithm 1, step 4), so a multi-GPU run gives each rank a disjoint range of global
chain indices. The Philox counter word 2 is the global chain index, so every chain's
trajectory is the same whichever rank runs it. The only exchange is one reduction of
per-chain results at the end, done here on the host through torch.distributed (gloo or
nccl); there is no collective on the data path.
"""
import math


def chain_range(rank, world, total_chains):
    """Contiguous [offset, offset + count) of global chain indices for `rank` (strong
    partition of a fixed total; the first `total % world` ranks get one extra)."""
    if world < 1 or not 0 <= rank < world or total_chains < 0:
        raise ValueError("bad rank/world/total")
    base, extra = divmod(total_chains, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def weak_offset(rank, chains_per_rank):
    """Global index of a rank's first chain when every rank runs the same count."""
    return rank * chains_per_rank


def pool(per_chain):
    """Pool per-chain means {key: [values]} into (mean, standard error across chains)."""
    out = {}
    for k, vals in per_chain.items():
        n = len(vals)
        m = sum(vals) / n
        err = math.sqrt(sum((v - m) ** 2 for v in vals) / (n - 1) / n) if n > 1 else 0.0
        out[k] = (m, err)
    return out


def gather_per_chain(local, offset, dist=None):
    """All ranks: gather {key: [per-chain values]} of every rank, ordered by global chain
    index, so that pooling sees exactly what a single process would."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    items = [None] * dist.get_world_size()
    dist.all_gather_object(items, (offset, local))
    items.sort(key=lambda t: t[0])
    merged = {}
    for _, d in items:
        for k, v in d.items():
            merged.setdefault(k, []).extend(v)
    return merged


def max_over_ranks(value, dist=None):
    """Maximum of a host float over ranks (the timing rule: slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
