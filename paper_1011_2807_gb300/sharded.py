"""S-sharded join across ranks, one GPU each: every rank holds the index of one range
of S, joins the same queries against it, and the ranks exchange their per-row top-k
lists (all-gather) and merge them into the top-k of the whole S (``knn_merge_topk``).
This is Algorithm 1's loop over S blocks split across GPUs, plus the exchange step
that the split needs; the same merge serves an S joined range by range on one GPU.

Only the exchange lives here; the join and the merge are the library's calls.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import binding


def shard_range(n_s: int, rank: int, world: int) -> tuple[int, int]:
    """The rows [a, b) of S that `rank` of `world` holds: contiguous ranges whose sizes
    differ by at most one."""
    base, extra = divmod(int(n_s), int(world))
    a = rank * base + min(rank, extra)
    return a, a + base + (1 if rank < extra else 0)


def knn_join_sharded(index, R, k: int, s_offset: int, *, group=None, join=None, merge=None, **join_kw):
    """Top-k of every row of R over the whole S, on every rank of `group`.

    ``index`` is this rank's index (of S rows starting at ``s_offset``); the result's ids
    are global.  ``join`` and ``merge`` default to ``binding.knn_join`` and
    ``binding.knn_merge_topk``; keyword arguments go to the join.  With NCCL the
    exchanged tensors are the join's device outputs.
    """
    join = join or binding.knn_join
    merge = merge or binding.knn_merge_topk
    ids, sc = join(index, R, k, **join_kw)
    ids, sc = ids.contiguous(), sc.contiguous()
    world = dist.get_world_size(group)
    all_ids = [torch.empty_like(ids) for _ in range(world)]
    all_sc = [torch.empty_like(sc) for _ in range(world)]
    dist.all_gather(all_ids, ids, group=group)
    dist.all_gather(all_sc, sc, group=group)
    off = torch.tensor([int(s_offset)], dtype=torch.int64, device=ids.device)
    all_off = [torch.empty_like(off) for _ in range(world)]
    dist.all_gather(all_off, off, group=group)
    return merge(list(zip(all_ids, all_sc)), [int(o.item()) for o in all_off], k)
