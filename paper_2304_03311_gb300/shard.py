"""Trajectory sharding across ranks and the one exchange step of the method.

Trajectories of a transformation are independent and the global trajectory
index is part of every random counter, so any split of the index range over
ranks reproduces the single-process run bit for bit.  The only data exchange
is gathering the int64 W_int arrays (8 bytes per trajectory) before the
estimator; the gathered array is in global trajectory order, so the estimator
sees exactly the array a single process would have produced.

Failure detection is on the host: a rank that dies or never joins makes the
collective fail within the process group's timeout, and ``merge_shards``
rejects a gather with a missing or mis-sized shard.
"""
from __future__ import annotations

import numpy as np


class MissingShardError(RuntimeError):
    """A rank's share of the trajectories did not arrive."""


def shard_range(n_traj: int, rank: int, world: int, traj0: int = 0):
    """(first global trajectory, count) of rank's contiguous share; the first
    n_traj % world ranks get one extra trajectory."""
    if world < 1 or not 0 <= rank < world or n_traj < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_traj, world)
    count = base + (1 if rank < extra else 0)
    first = traj0 + rank * base + min(rank, extra)
    return first, count


def merge_shards(parts, n_traj: int, world: int) -> np.ndarray:
    """Concatenate per-rank W_int arrays (dict rank -> array or a list in rank
    order) in global trajectory order, checking every shard is present and has
    its expected length."""
    if isinstance(parts, dict):
        missing = [r for r in range(world) if r not in parts]
        if missing:
            raise MissingShardError(f"no work from ranks {missing}")
        parts = [parts[r] for r in range(world)]
    if len(parts) != world:
        raise MissingShardError(f"{len(parts)} shards for {world} ranks")
    out = []
    for r, a in enumerate(parts):
        want = shard_range(n_traj, r, world)[1]
        a = np.asarray(a, dtype=np.int64).reshape(-1)
        if a.size != want:
            raise MissingShardError(f"rank {r} sent {a.size} trajectories, expected {want}")
        out.append(a)
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


def gather_work(local, n_traj: int, group=None) -> np.ndarray:
    """All-gather the ranks' W_int shards (torch.distributed, any backend) and
    merge them in global order.  Raises MissingShardError when a rank's share
    is absent or the collective fails (a dead rank surfaces as a timeout)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    want = shard_range(n_traj, rank, world)[1]
    local = np.asarray(local, dtype=np.int64).reshape(-1)
    if local.size != want:
        raise MissingShardError(f"rank {rank} holds {local.size} trajectories, expected {want}")
    size = shard_range(n_traj, 0, world)[1]
    buf = torch.zeros(size, dtype=torch.int64)
    buf[:local.size] = torch.from_numpy(local)
    parts = [torch.zeros(size, dtype=torch.int64) for _ in range(world)]
    try:
        dist.all_gather(parts, buf, group=group)
    except Exception as exc:   # a peer died or timed out
        raise MissingShardError(f"gather failed: {exc}") from exc
    return merge_shards([p[:shard_range(n_traj, r, world)[1]].numpy() for r, p in enumerate(parts)],
                        n_traj, world)
