"""Sharding of the search over several GPUs (one process each) or calls.

The path splits into independent units that exchange nothing but their
top-K lists: the trajectories of one map's grid (ranges of the trajectory
index), and the (s, q) maps of a sweep.  Each shard runs the library's own
search on its device; the lists (top_k records of 72 bytes each) are
gathered and merged on the host, the merge being morse_topk_merge on the
key (chi^2, idx).  A trajectory's chi^2 does not depend on the shard that
computes it, so the merged list equals the unsharded one bit for bit.

Gathering is the caller's: a function that takes this shard's result and
returns every shard's, in rank order -- ``torch_gather()`` over
torch.distributed (NCCL or gloo), or ``LocalGather`` when the shards run
one after the other in one process.
"""
from __future__ import annotations

import numpy as np

from . import FIT_DTYPE, topk_merge


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """(first, count) of shard `rank` of `world` contiguous shards of n
    units (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    first = rank * n // world
    return first, (rank + 1) * n // world - first


def empty_fits(k: int) -> np.ndarray:
    """A top-K list with no entry (idx -1, chi^2 +inf)."""
    out = np.zeros(k, dtype=FIT_DTYPE)
    out["chi2"] = np.inf
    out["idx"] = -1
    return out


def sharded_topk(search_range, n: int, k: int, rank: int, world: int,
                 gather) -> np.ndarray:
    """The top-k of n trajectories split over `world` shards: this shard
    runs search_range(first, count) on its range, the lists are gathered and
    merged.  Every rank returns the same merged list."""
    first, count = shard_range(n, rank, world)
    mine = search_range(first, count) if count > 0 else empty_fits(k)
    return topk_merge(gather(np.ascontiguousarray(mine, dtype=FIT_DTYPE)),
                      k)


def search(ctx, event, map_, grid, rank: int, world: int,
           gather) -> np.ndarray:
    """One map's grid search (morse_grid_chi2) split by trajectory index:
    this rank searches its range with morse_grid_chi2_range on ctx's
    device; returns the merged top-K (equal to morse_grid_chi2's)."""
    return sharded_topk(
        lambda f, c: ctx.grid_chi2_range(event, map_, grid, f, c),
        grid.size, grid.top_k, rank, world, gather)


def sweep(ctx, event, s, q, extent, npix, rays_per_axis, grid, rank: int,
          world: int, gather, **map_opts) -> np.ndarray:
    """The (s, q) sweep (morse_sweep) split by map: this rank builds and
    searches its contiguous block of the maps; returns every map's top-K
    list in map order, [n_maps, top_k] (equal to morse_sweep's)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    first, count = shard_range(len(s), rank, world)
    if count > 0:
        mine = ctx.sweep(event, s[first:first + count].copy(),
                         q[first:first + count].copy(), extent, npix,
                         rays_per_axis, grid, **map_opts)
    else:
        mine = np.zeros((0, grid.top_k), dtype=FIT_DTYPE)
    parts = gather(mine)
    return np.concatenate([np.asarray(p, dtype=FIT_DTYPE).reshape(
        -1, grid.top_k) for p in parts])


def best_over_maps(lists: np.ndarray, k: int):
    """The k best records over all maps of a sweep: (map index, record)
    pairs ordered by (chi^2, map, idx)."""
    lists = np.asarray(lists, dtype=FIT_DTYPE)
    maps = np.repeat(np.arange(lists.shape[0]), lists.shape[1])
    flat = lists.reshape(-1)
    keep = flat["idx"] >= 0
    order = np.lexsort((flat["idx"][keep], maps[keep], flat["chi2"][keep]))
    sel = order[:k]
    return maps[keep][sel], flat[keep][sel]


class LocalGather:
    """Gather for shards run one after the other in one process, in rank
    order: each call returns the results so far, so the last rank's call
    sees every shard's."""

    def __init__(self):
        self._parts = []

    def __call__(self, mine):
        self._parts.append(mine)
        return list(self._parts)


def torch_gather(group=None):
    """A gather over torch.distributed: every rank's result, in rank order
    (all_gather_object; results are small host arrays)."""
    import torch.distributed as dist

    def gather(mine):
        world = dist.get_world_size(group)
        parts = [None] * world
        dist.all_gather_object(parts, mine, group=group)
        return parts
    return gather
