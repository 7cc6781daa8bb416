"""Sharded search (database sharding: every query searches every shard, then one
merge of the shards' top-k lists by (distance, global id)).

* the oracle's merge is pinned against sorting the union of the lists;
* the multi-rank orchestration (all-gather of each rank's results and id offset, then merge)
  runs on CPU ranks over gloo, with the oracle's merge;
* on the GPU, three logical shards merged by lc_merge_topk equal the oracle's per-shard search
  followed by the oracle's merge.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_09996_gb300 import shard


def test_oracle_merge_is_sorted_union(rng):
    S, nq, k = 3, 5, 4
    ids = rng.integers(0, 100, size=(S, nq, k)).astype(np.int32)
    ds = rng.random((S, nq, k))
    ids[1, 2, 3] = -1
    offs = [0, 100, 200]
    mi, md = oracle.merge_topk(ids, ds, offs, k)
    for q in range(nq):
        union = sorted((ds[s, q, j], ids[s, q, j] + offs[s]) for s in range(S) for j in range(k) if ids[s, q, j] >= 0)
        assert [u[1] for u in union[:k]] == mi[q].tolist()
        assert np.allclose([u[0] for u in union[:k]], md[q])


def _rank_main(rank, ws, port, ids, ds, offs, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)

    def cpu_merge(i, d, o, k):
        mi, md = oracle.merge_topk(i.numpy(), d.numpy(), o, k)
        return torch.from_numpy(mi), torch.from_numpy(md)

    mi, md = shard.gather_and_merge(torch.from_numpy(ids[rank]), torch.from_numpy(ds[rank]), offs[rank],
                                    merge=cpu_merge)
    out.put((rank, mi.numpy(), md.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_and_merge_two_ranks_gloo(rng):
    import socket

    import torch.multiprocessing as mp
    ws, nq, k = 2, 6, 5
    ids = [np.sort(rng.choice(500, size=(nq, k)), axis=1).astype(np.int32) for _ in range(ws)]
    ds = [np.sort(rng.random((nq, k)), axis=1).astype(np.float32) for _ in range(ws)]
    offs = [0, 500]
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, ids, ds, offs, out)) for r in range(ws)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref_i, ref_d = oracle.merge_topk(np.stack(ids), np.stack(ds), offs, k)
    for rank, mi, md in got:
        assert np.array_equal(mi, ref_i)
        assert np.allclose(md, ref_d)


@pytest.mark.gpu
def test_logical_shards_match_oracle_per_shard_and_merge():
    import torch

    from paper_1804_09996_gb300 import build, datagen as dg, lc
    build.build()
    xt = dg.gaussian_mixture(4000, 96, 64, stream=dg.STREAM_TRAIN)
    xb = dg.gaussian_mixture(2400, 96, 64, stream=dg.STREAM_BASE)
    xq = dg.gaussian_mixture(120, 96, 64, stream=dg.STREAM_QUERY)
    ranges = shard.split_ranges(len(xb), 3)
    k, ef = 10, 48
    handles, refs, gaps = [], [], []
    for a, b in ranges:
        ix = oracle.build_index(xt, xb[a:b], 16, 16, False, codec_niter=8)
        h = lc.lc_create(lc.lc_default_params(96, 16, 16))
        lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0,
                     ix.levels, ix.upper_adj, ix.ep)
        handles.append(h)
        r = oracle.search(ix, xq, k, ef)
        refs.append(r)
        gaps.append(r["gap"])
    try:
        sh = shard.LogicalShards(handles, [a for a, _ in ranges])
        q = torch.from_numpy(xq).cuda()
        gi, gd = sh.search(q, len(xq), lc.lc_default_search_params(k, ef))
        torch.cuda.synchronize()
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    finally:
        for h in handles:
            lc.lc_free(h)
    ri, rd = oracle.merge_topk(np.stack([r["ids"] for r in refs]), np.stack([r["dists"] for r in refs]),
                               [a for a, _ in ranges], k)
    # exempt queries with a near-tie in any shard, or between adjacent merged results
    rel = np.diff(rd, axis=1) / rd[:, 1:]
    ok = (np.min(np.stack(gaps), axis=0) >= 1e-6) & (np.nan_to_num(rel, nan=1.0).min(axis=1) >= 1e-6)
    assert ok.mean() > 0.8
    assert np.array_equal(gi[ok], ri[ok])
    fin = np.isfinite(rd[ok])
    np.testing.assert_allclose(gd[ok][fin], rd[ok][fin], rtol=1e-5)
