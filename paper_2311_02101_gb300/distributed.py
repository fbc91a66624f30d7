"""Chain sharding across ranks (one process per GPU).

Chains are independent Markov chains (Sec. 4.2), so a run of B chains per rank
on N ranks is one ensemble of N * B chains: rank r runs the global chains
r * B .. r * B + B - 1 (maxsat_reset_shard), whose draws and temperatures follow
their global index. The only exchange is at the end: the lowest cost over all
ranks (ties to the lowest global chain index) and its assignment.
"""
from __future__ import annotations

import numpy as np


def shard_of(rank: int, world: int, chains_per_rank: int):
    """(chain_offset, total_chains) of a rank; chains_per_rank must be a
    multiple of 8 (draw counters group chains by 8)."""
    if chains_per_rank % 8:
        raise ValueError("chains per rank must be a multiple of 8")
    return rank * chains_per_rank, world * chains_per_rank


def reduce_best(cost: int, chain: int, assignment: np.ndarray, group=None, device=None):
    """Global best over all ranks: every rank passes its best cost, the global
    index of the chain that reached it and that chain's assignment (uint8,
    length n). Returns (cost, chain, assignment) of the lowest cost, ties to
    the lowest chain index, on every rank. One all-gather of two integers and
    one broadcast of n bytes."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = device or ("cuda" if dist.get_backend(group) == "nccl" else "cpu")
    mine = torch.tensor([int(cost), int(chain)], dtype=torch.int64, device=dev)
    every = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    pairs = [(int(t[0]), int(t[1]), r) for r, t in enumerate(every)]
    best_cost, best_chain, owner = min(pairs)
    buf = torch.from_numpy(np.ascontiguousarray(assignment, np.uint8)).to(dev)
    dist.broadcast(buf, src=dist.get_global_rank(group, owner) if group is not None else owner,
                   group=group)
    return best_cost, best_chain, buf.cpu().numpy()
