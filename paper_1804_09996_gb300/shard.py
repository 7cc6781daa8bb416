"""Sharded search: a database split into S contiguous id ranges, one Link-and-Code index per
shard.  Every query searches every shard, and the shards' top-k lists are merged by
(distance, global id) with lc_merge_topk (global id = shard-local id + the shard's first id).

* LogicalShards: all shards on one GPU (an index larger than one graph should be, or a test
  of the multi-GPU path on a single device).
* gather_and_merge: one shard per rank; the only data exchange is an all-gather of every
  rank's [nq][k] (id, distance) results and id offsets, followed by the merge.

Argument marshalling and orchestration only: the searches and the merge run in liblc.so.
"""
from __future__ import annotations

import numpy as np

from . import lc


class LogicalShards:
    """Several indexes on the current GPU, searched together."""

    def __init__(self, handles, offsets):
        if len(handles) != len(offsets) or not handles:
            raise ValueError("one id offset per shard")
        self.handles = list(handles)
        self.offsets = [int(o) for o in offsets]

    def search(self, q, nq: int, sp, stream=None):
        """q: device float32 tensor [nq][d].  Returns device (ids [nq][k], dists [nq][k])."""
        import torch
        S, k = len(self.handles), sp.k
        ids = torch.empty((S, nq, k), dtype=torch.int32, device=q.device)
        ds = torch.empty((S, nq, k), dtype=torch.float32, device=q.device)
        for s, h in enumerate(self.handles):
            lc.lc_search(h, q, nq, sp, ids[s], ds[s], None, stream)
        out_i = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        out_d = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        lc.lc_merge_topk(ids, ds, S, nq, k, self.offsets, out_i, out_d, stream)
        return out_i, out_d


def gpu_merge(ids, dists, offsets, k):
    """lc_merge_topk on stacked device tensors [S][nq][k]."""
    import torch
    S, nq = ids.shape[0], ids.shape[1]
    out_i = torch.empty((nq, k), dtype=torch.int32, device=ids.device)
    out_d = torch.empty((nq, k), dtype=torch.float32, device=ids.device)
    lc.lc_merge_topk(ids.contiguous(), dists.contiguous(), S, nq, k, offsets, out_i, out_d)
    return out_i, out_d


def gather_and_merge(ids_local, dists_local, offset: int, group=None, merge=gpu_merge):
    """Rank-sharded search: all-gather each rank's local results ([nq][k] tensors on the
    collective's device) and id offset, then merge them into global top-k lists.  `merge`
    takes (ids [S][nq][k], dists [S][nq][k], offsets list, k)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    ids_all = [torch.empty_like(ids_local) for _ in range(ws)]
    ds_all = [torch.empty_like(dists_local) for _ in range(ws)]
    off_all = [torch.zeros(1, dtype=torch.int64, device=ids_local.device) for _ in range(ws)]
    dist.all_gather(ids_all, ids_local.contiguous(), group=group)
    dist.all_gather(ds_all, dists_local.contiguous(), group=group)
    dist.all_gather(off_all, torch.tensor([offset], dtype=torch.int64, device=ids_local.device), group=group)
    offsets = [int(o.item()) for o in off_all]
    return merge(torch.stack(ids_all), torch.stack(ds_all), offsets, ids_local.shape[1])


def split_ranges(n: int, shards: int):
    """Contiguous id ranges [(start, stop)] of near-equal size."""
    b = np.linspace(0, n, shards + 1).astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(shards)]
