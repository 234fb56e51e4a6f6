"""Splitting one batch of environments over several GPUs (one process each).

Environments are independent (Sec. 3.1 "Batching": every environment is
stepped by the same simulator, with no interaction between them), so a batch
of N environments splits into G contiguous shards with no exchange on the
data path: rank g steps environments [g*N/G, (g+1)*N/G) and holds only the
scenes those environments use.  A shard's context gets ``env_offset`` = its
first global index, so its resets and placing jitters draw the Philox
counters of the global environment indices, and every environment evolves
exactly as it would in one context over the whole batch.  Per-step counters
(rewards, contacts, events) are summed across ranks on the host.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs as _inputs


def env_range(n_global: int, world: int, rank: int) -> tuple[int, int]:
    """First global environment and count of rank `rank`'s shard:
    [rank*N/world, (rank+1)*N/world) with integer floor division, so the
    shards partition [0, N) and differ in size by at most one."""
    if not (0 <= rank < world) or n_global < world:
        raise ValueError("need 0 <= rank < world <= n_global")
    first = rank * n_global // world
    last = (rank + 1) * n_global // world
    return first, last - first


@dataclasses.dataclass(frozen=True)
class ShardPlan:
    rank: int
    world: int
    first: int                 # global index of the shard's environment 0
    count: int                 # environments in the shard
    scenes: tuple[int, ...]    # global scene indices the shard loads, ascending
    env_scene: np.ndarray      # [count] local scene index (into `scenes`) per environment


def plan(n_global: int, n_scenes: int, world: int, rank: int,
         env_scene_global: np.ndarray | None = None) -> ShardPlan:
    """The shard of `rank`: its environment range, the global scenes its
    environments use (and no other) and its environments' scene map into
    that subset.  env_scene_global: [n_global] scene per environment, default
    the contiguous blocks env i -> floor(i * n_scenes / n_global)."""
    gmap = (_inputs.env_scene_map(n_global, n_scenes) if env_scene_global is None
            else np.asarray(env_scene_global, np.int64))
    if len(gmap) != n_global:
        raise ValueError("env_scene_global must have n_global entries")
    first, count = env_range(n_global, world, rank)
    mine = gmap[first:first + count]
    used = tuple(int(s) for s in np.unique(mine))
    local = np.searchsorted(np.asarray(used), mine).astype(np.int32)
    return ShardPlan(rank, world, first, count, used, local)


def sum_counters(dist, values: dict[str, float]) -> dict[str, float]:
    """Host-side sum of per-rank counters over all ranks (a CPU tensor
    all-reduce: with NCCL ranks it goes through a gloo group the caller
    made, passed as dist=(torch.distributed, group))."""
    import torch
    if dist is None:
        return dict(values)
    d, group = dist if isinstance(dist, tuple) else (dist, None)
    keys = sorted(values)
    t = torch.tensor([float(values[k]) for k in keys], dtype=torch.float64)
    d.all_reduce(t, op=d.ReduceOp.SUM, group=group)
    return {k: float(v) for k, v in zip(keys, t.tolist())}
