"""Table-sharded search over several processes (one GPU each).

Every rank holds an index over the same points built from the same seed and
searches only its slice of the tables (``fpp_search_ex`` with a table
range); the ranks' top-k lists are all-gathered and merged with
``fpp_merge_topk``.  The exact top-k over the union of all tables'
candidates lies in the union of the per-slice top-k lists, so the merged
result equals the unsharded search.  The only exchange is the all-gather of
k (id, score) pairs per query.
"""
from __future__ import annotations

import numpy as np

from . import fpp_merge_topk, fpp_search_ex


def table_range(rank: int, world: int, L: int) -> tuple[int, int]:
    """Tables [begin, end) of a rank: contiguous slices differing by at most one."""
    if not 0 <= rank < world or L < world:
        raise ValueError("need 0 <= rank < world <= L")
    base, extra = divmod(L, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_merge(local_ids, local_scores, group=None):
    """All-gathers every rank's [m][k] top-k lists (host arrays) over the
    process group and merges them into the global [m][k] top-k."""
    import torch
    import torch.distributed as dist

    ids = torch.from_numpy(np.ascontiguousarray(local_ids, dtype=np.int64))
    sc = torch.from_numpy(np.ascontiguousarray(local_scores, dtype=np.float32))
    world = dist.get_world_size(group)
    all_ids = [torch.empty_like(ids) for _ in range(world)]
    all_sc = [torch.empty_like(sc) for _ in range(world)]
    dist.all_gather(all_ids, ids, group=group)
    dist.all_gather(all_sc, sc, group=group)
    return fpp_merge_topk(torch.stack(all_ids).numpy(), torch.stack(all_sc).numpy())


def sharded_search(index, Q, k: int, probes: int, group=None):
    """Searches this rank's slice of the tables of ``index`` and returns the
    merged global top-k ([m][k] host arrays) on every rank."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    L = index.info()["L"]
    tb, te = table_range(rank, world, L)
    ids, scores, _ = fpp_search_ex(index.handle, Q, k=k, probes=probes, table_begin=tb,
                                   table_end=te, want_stats=False)
    if not isinstance(ids, np.ndarray):
        ids, scores = ids.cpu().numpy(), scores.cpu().numpy()
    return gather_merge(ids, scores, group)
