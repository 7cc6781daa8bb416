"""Search of the oracle (wrapper of ``orc_search`` in lc_oracle.c) and brute-force k-NN.

Test infrastructure only (see the package docstring).

The search follows Section 4.1's two-stage strategy over the HNSW structure of Section 2:
the walk scores database vectors by ADC from their level-1 codes, and the shortlist of the
best walk results is re-ranked with the refined reconstruction beta_b^T G(x) of Section 4.3
(q = c1 + c2 being the two-level decoding).  ``shortlist`` = 0 refines max(k, 10) vectors
(Section 5.1, "at most 10" when k <= 10), a positive value refines max(shortlist, k), and a
negative value skips the refinement and returns the walk's own top-k.
"""
from __future__ import annotations

import numpy as np

from ._clib import lib, ptr


def search(ix, Q: np.ndarray, k: int, ef: int, shortlist: int = 0, return_w: bool = False,
           beam: int = 1, tcap: int = 0, c1_walk: np.ndarray | None = None, walk_full: bool = False,
           c2_walk: np.ndarray | None = None):
    """Returns dict(ids [nq][k] int32, dists [nq][k] float64, stats [nq][3] int32 =
    (n_dist, n_expand, n_dist_upper), gap [nq] = smallest relative gap of a deciding
    comparison, gap_walk [nq] = the same over the comparisons that decide the walk and the
    shortlist (not the order of the k returned), next_dist [nq] = the distance that follows
    the k returned in the list they were taken from (+inf if none), ctx = the arguments that
    ``dists`` needs to recompute any returned id's distance, and with ``return_w`` the final
    result set W sorted by (dist, id)).  ``beam``
    >= 2 selects the batched form of the level-0 search (that many expansions per step);
    ``tcap`` > 0 stops the level-0 search once that many distances were computed (Section 3.1's
    search-time parameter T, checked before each expansion).  ``c1_walk`` replaces the level-1
    codebook in the walk's ADC terms only (e.g. C1 rounded to FP16); the re-rank uses ix.C1.
    ``walk_full`` makes the walk score the full two-level decode q = c1 + c2 (Section 4.1's
    approximation taken in full) instead of the level-1 code; ``c2_walk`` then replaces C2 in
    the walk as ``c1_walk`` replaces C1."""
    Q = np.ascontiguousarray(Q, np.float32)
    nq = Q.shape[0]
    efp = max(ef, k)
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    stats = np.empty((nq, 3), np.int32)
    gap = np.empty(nq, np.float64)
    gap_walk = np.empty(nq, np.float64)
    next_dist = np.empty(nq, np.float64)
    w_ids = np.empty((nq, efp), np.int32) if return_w else None
    w_d = np.empty((nq, efp), np.float64) if return_w else None
    w_n = np.empty(nq, np.int32) if return_w else None
    N = ix.codes1.shape[0]
    rc = lib().orc_search(
        N, ix.d, ix.M1, ix.M2, ptr(ix.R), ptr(ix.C1), ptr(ix.C2), ptr(ix.codes1),
        ptr(ix.codes2), ptr(np.ascontiguousarray(ix.beta, np.uint8)), ptr(np.ascontiguousarray(ix.B, np.float32)),
        getattr(ix, "bM", 1), getattr(ix, "bK", 256), ix.adj0.shape[1], ptr(ix.adj0),
        ix.upper_adj.shape[1], ptr(ix.upper_off),
        ptr(ix.upper_adj) if ix.upper_adj.shape[0] > 0 else None, ix.ep, ix.max_level,
        nq, ptr(Q), k, ef, shortlist, beam, tcap,
        ptr(np.ascontiguousarray(c1_walk, np.float32)) if c1_walk is not None else None, int(walk_full),
        ptr(np.ascontiguousarray(c2_walk, np.float32)) if c2_walk is not None else None,
        ptr(ids), ptr(dists), ptr(stats), ptr(gap), ptr(gap_walk), ptr(next_dist),
        ptr(w_ids), ptr(w_d), ptr(w_n))
    if rc != 0:
        raise RuntimeError(f"orc_search failed ({rc})")
    out = dict(ids=ids, dists=dists, stats=stats, gap=gap, gap_walk=gap_walk, next_dist=next_dist,
               ctx=dict(ix=ix, Q=Q, shortlist=shortlist, c1_walk=c1_walk, walk_full=walk_full, c2_walk=c2_walk))
    if return_w:
        out.update(w_ids=w_ids, w_dists=w_d, w_size=w_n)
    return out


def dists(ix, Q: np.ndarray, ids: np.ndarray, c1_walk: np.ndarray | None = None, walk_full: bool = False,
          c2_walk: np.ndarray | None = None):
    """The walk distance and the refined distance of given ids [nq][m] (-1: +inf) for each
    query, computed directly from their definitions (rotation, ADC sum or full decode,
    refined reconstruction of Section 4.3), without any walk.  ``c1_walk``, ``walk_full`` and
    ``c2_walk`` as in ``search``.  Returns (walk [nq][m], refined [nq][m]) float64."""
    Q = np.ascontiguousarray(Q, np.float32)
    ids = np.ascontiguousarray(ids, np.int32)
    nq, m = ids.shape
    walk = np.empty((nq, m), np.float64)
    ref = np.empty((nq, m), np.float64)
    N = ix.codes1.shape[0]
    rc = lib().orc_dists(
        N, ix.d, ix.M1, ix.M2, ptr(ix.R), ptr(ix.C1), ptr(ix.C2), ptr(ix.codes1),
        ptr(ix.codes2), ptr(np.ascontiguousarray(ix.beta, np.uint8)), ptr(np.ascontiguousarray(ix.B, np.float32)),
        getattr(ix, "bM", 1), getattr(ix, "bK", 256), ix.adj0.shape[1], ptr(ix.adj0),
        nq, ptr(Q), m, ptr(ids),
        ptr(np.ascontiguousarray(c1_walk, np.float32)) if c1_walk is not None else None, int(walk_full),
        ptr(np.ascontiguousarray(c2_walk, np.float32)) if c2_walk is not None else None,
        ptr(walk), ptr(ref))
    if rc != 0:
        raise RuntimeError(f"orc_dists failed ({rc})")
    return walk, ref


# kinds of deciding comparison reported by ``trace`` (lc_oracle.c)
GAP_KINDS = {1: "upper_second", 2: "upper_move", 3: "runner", 4: "outside", 5: "break", 6: "end",
             7: "batch_next", 8: "batch_outside", 9: "batch_end", 10: "shortlist", 11: "out_walk",
             12: "out_refined"}


def trace(fn, cap: int = 1 << 16):
    """Runs ``fn()`` (oracle searches on this thread) and returns (its result, the list of
    deciding comparisons it recorded, in order, as (kind name, id, id) triples)."""
    buf = np.zeros((cap, 3), np.int32)
    lib().orc_trace(ptr(buf), cap)
    try:
        out = fn()
    finally:
        n = lib().orc_trace(None, 0)
    return out, [(GAP_KINDS[int(a)], int(b), int(c)) for a, b, c in buf[:n]]


def merge_topk(ids: np.ndarray, dists: np.ndarray, offsets, k: int):
    """Merged top-k of per-shard results [S][nq][k] by (distance, global id), global id =
    local id + the shard's offset; -1 entries are padding.  Returns (ids [nq][k] int64,
    dists [nq][k] float64)."""
    S, nq, _ = ids.shape
    out_i = np.full((nq, k), -1, np.int64)
    out_d = np.full((nq, k), np.inf)
    for q in range(nq):
        cand = [(float(dists[s, q, j]), int(ids[s, q, j]) + int(offsets[s]))
                for s in range(S) for j in range(ids.shape[2]) if ids[s, q, j] >= 0]
        cand.sort()
        for j, (d, i) in enumerate(cand[:k]):
            out_i[q, j], out_d[q, j] = i, d
    return out_i, out_d


def knn(X: np.ndarray, Q: np.ndarray, k: int, chunk: int = 256):
    """Exact k nearest neighbours of each query in X under squared L2, float64, by
    exhaustive comparison (Section 2's problem statement).  Ties go to the smaller id."""
    X = np.asarray(X, np.float64)
    Q = np.asarray(Q, np.float64)
    ids = np.empty((Q.shape[0], k), np.int64)
    ds = np.empty((Q.shape[0], k))
    for a in range(0, Q.shape[0], chunk):
        q = Q[a:a + chunk]
        D = np.empty((q.shape[0], X.shape[0]))
        for b in range(0, X.shape[0], 65536):
            diff = q[:, None, :] - X[None, b:b + 65536, :]
            D[:, b:b + 65536] = np.einsum("qnd,qnd->qn", diff, diff)
        order = np.lexsort((np.broadcast_to(np.arange(X.shape[0]), D.shape), D), axis=1)[:, :k]
        ids[a:a + chunk] = order
        ds[a:a + chunk] = np.take_along_axis(D, order, axis=1)
    return ids, ds
