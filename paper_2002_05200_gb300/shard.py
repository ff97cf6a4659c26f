"""Multi-GPU sharding of a batch of independent pairs (host side only).

The paper's balancer (Sec. IV-C) splits the alignments across GPUs by count
and sequence length, lets each GPU run its share independently and gathers
the results on the host.  Pairs never exchange data, so there is no
collective on the data path: only the host-side gather of results and the
timing reduction use torch.distributed.

* ``lpt_partition``: longest-processing-time assignment of pairs to ranks by
  estimated work (sum of the two sequence lengths).
* ``shard_indices``: this rank's pair indices (sorted, so each shard keeps
  input order); ``shard_batch``: the batch restricted to them.
* ``gather_results``: reassembles per-rank result arrays in input order on
  every rank.
* ``reduce_step``: max of the step time and sum of the cells over ranks.
"""
from __future__ import annotations

import heapq

import numpy as np


def pair_work(b) -> np.ndarray:
    """Work estimate per pair: bases of A plus bases of B (anti-diagonals of
    the two extensions together)."""
    s = b.seeds
    return b.lenA[s["idxA"]].astype(np.int64) + b.lenB[s["idxB"]].astype(np.int64)


def lpt_partition(work: np.ndarray, world: int):
    """Assigns each item to the least-loaded rank, largest items first.
    Returns a list of `world` sorted index arrays covering every item once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-np.asarray(work, dtype=np.int64), kind="stable")
    heap = [(0, r) for r in range(world)]
    owner = np.empty(len(order), dtype=np.int64)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(work[i]), r))
    return [np.flatnonzero(owner == r) for r in range(world)]


def shard_indices(b, world: int, rank: int) -> np.ndarray:
    return lpt_partition(pair_work(b), world)[rank]


def shard_batch(b, idx: np.ndarray):
    """This rank's pairs as a batch of its own: the same sequence pools (each
    rank holds the whole read set), the seeds and per-pair X of `idx` only."""
    import dataclasses
    return dataclasses.replace(b, seeds=b.seeds[idx].copy(),
                               Xs=None if b.Xs is None else b.Xs[idx].copy(),
                               name=f"{b.name}[shard]")


def gather_results(local: np.ndarray, idx: np.ndarray, n_total: int, group=None) -> np.ndarray:
    """All ranks' (indices, results) -> one array in input order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (np.asarray(idx), np.asarray(local)), group=group)
    out = np.zeros(n_total, dtype=local.dtype)
    seen = np.zeros(n_total, dtype=bool)
    for ii, rr in parts:
        if seen[ii].any():
            raise RuntimeError("a pair was computed by two ranks")
        out[ii] = rr
        seen[ii] = True
    if not seen.all():
        raise RuntimeError("some pairs were computed by no rank")
    return out


def reduce_step(ms: float, cells: int, device="cpu", group=None):
    """(max ms over ranks, total cells over ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), int(c.item())
