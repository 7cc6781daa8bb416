"""Pins for the oracle's graph build (Section 2, 4.1, 5.1): level draws (SplitMix64 against
its published outputs, geometric sizes with ratio 30), structural invariants of the HNSW
rows, connectivity, the shrinking heuristic on a hand-worked case, and batched insertion."""
import math

import numpy as np

import oracle
from oracle import graph


def test_splitmix64_published_outputs():
    # first outputs of SplitMix64 for seeds 0 and 1234567 (reference implementation values)
    assert [int(v) for v in graph.splitmix64(0, np.arange(3))] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in graph.splitmix64(1234567, np.arange(3))] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_level_sizes_follow_ratio_30():
    lev = graph.levels(300_000, seed=1804)
    n1 = int((lev >= 1).sum())
    n2 = int((lev >= 2).sum())
    # P(level >= l) = 30^-l
    assert abs(n1 - 300_000 / 30) < 5 * math.sqrt(300_000 / 30)
    assert abs(n2 - 300_000 / 900) < 5 * math.sqrt(300_000 / 900)
    assert np.array_equal(graph.levels(10, 7, start=5), graph.levels(15, 7)[5:])


def check_structure(ix):
    N, deg = ix.adj0.shape
    xh = ix.extra["xh"]
    for i in range(N):
        row = ix.adj0[i]
        n = int((row >= 0).sum())
        assert (row[:n] >= 0).all() and (row[n:] == -1).all()
        assert i not in row[:n]
        assert len(set(row[:n].tolist())) == n
        d = ((xh[row[:n]] - xh[i]) ** 2).sum(1)
        # increasing distance to the owner (to float32 rounding for builds in float32)
        assert np.all(d[:-1] <= d[1:] * (1 + 1e-5) + 1e-12)
    lev = ix.levels
    assert lev[ix.ep] == lev.max() == ix.max_level
    for i in np.flatnonzero(lev > 0):
        for l in range(1, lev[i] + 1):
            row = ix.upper_adj[ix.upper_off[i] + l - 1]
            nb = row[row >= 0]
            assert (lev[nb] >= l).all()
    # level 0 is connected from the entry point
    seen, stack = {ix.ep}, [ix.ep]
    while stack:
        v = stack.pop()
        for e in ix.adj0[v]:
            if e >= 0 and e not in seen:
                seen.add(int(e))
                stack.append(int(e))
    assert len(seen) == N


def test_built_graph_invariants(mix3k):
    ix, _, _ = mix3k
    check_structure(ix)
    assert ix.adj0.shape[1] == 32
    assert (ix.adj0 >= 0).sum(1).mean() > 6


def test_heuristic_hand_case():
    # Points on a line at 0 (base, inserted last), 1, 2, 10.  Candidates by distance: 1 (1),
    # 2 (4), 10 (100).  Keep 1.  2 is closer to 1 (distance 1) than to the base (4): pruned.
    # 10 is closer to 2 (64)? 2 is not kept; compare with kept 1: (10-1)^2 = 81 < 100: pruned.
    # => the new node links to node 1 only, and node 1 gets a back-link.
    pts = np.array([[1.0], [2.0], [10.0], [0.0]])
    lev = np.zeros(4, np.int32)
    adj0, off, uadj, ep, ml = graph.build_graph(pts, pts, lev, deg=3, deg_up=3, efc=8, batch_max=1)
    assert adj0[3].tolist() == [0, -1, -1]
    assert 3 in adj0[0].tolist()


def test_sequential_and_batched_builds_both_work():
    from paper_1804_09996_gb300 import datagen as dg
    xt = dg.gaussian_mixture(3000, 96, 64, stream=dg.STREAM_TRAIN)
    xb = dg.gaussian_mixture(2000, 96, 64, stream=dg.STREAM_BASE)
    xq = dg.gaussian_mixture(200, 96, 64, stream=dg.STREAM_QUERY)
    gt, _ = oracle.knn(xb, xq, 1)
    rec = []
    for bm in (1, 64):
        ix = oracle.build_index(xt, xb, 16, 16, False, batch_max=bm)
        check_structure(ix)
        r = oracle.search(ix, xq, k=10, ef=64)
        rec.append((r["ids"] == gt).any(1).mean())
    assert min(rec) > 0.5 and abs(rec[0] - rec[1]) < 0.1
