"""GPU parity: the CUDA search path, called through the C ABI, against the FP64 oracle on
the same index (built by the oracle).

Bar (plain mode, FP32 tables), per query, by what the oracle's near-tie record says:
* no deciding comparison within 1e-6 relative: neighbour ids and visit counts (distinct nodes
  scored at level 0, level-0 expansions, upper-level evaluations) identical to the oracle's,
  returned distances within 1e-5 relative;
* near-ties only in the order of the k returned (the walk and the shortlist are decided):
  visit counts identical, ids identical at every position outside a run of near-tied
  distances, distances within 1e-5 relative position by position;
* every query, near-tie exempt or not: a valid result list (distinct ids, ascending by
  (distance, id), padding only at the end) whose every distance is the oracle's distance for
  that id, recomputed directly (ADC sum or refined reconstruction), within 1e-5 relative;
  over the batch, the GPU returns all but at most 0.5 % of the oracle's ids.
The share of exempt queries is bounded per test.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1804_09996_gb300 import lc

pytestmark = pytest.mark.gpu
TIE = 1e-6
RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1804_09996_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


_handles = {}


def handle(name, ix):
    if name not in _handles:
        h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2))
        lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0,
                     ix.levels, ix.upper_adj, ix.ep)
        _handles[name] = h
    return _handles[name]


def gpu_search(h, xq, k, ef, shortlist=0, device=True, visited_log=0, beam=1, tcap=0, lut_prec=0, walk_full=0):
    import torch
    nq = len(xq)
    sp = lc.lc_default_search_params(k, ef, shortlist=shortlist, visited_log=visited_log, max_dist=tcap,
                                     lut_prec=lut_prec, walk_full=walk_full)
    if beam > 1:
        sp.mode, sp.beam = lc.LC_MODE_BATCHED, beam
    if device:
        q = torch.from_numpy(np.ascontiguousarray(xq, np.float32)).cuda()
        ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
        ds = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
        st = torch.full((nq, 3), -7, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        lc.lc_search(h, q, nq, sp, ids, ds, st, s)
        s.synchronize()
        return ids.cpu().numpy(), ds.cpu().numpy(), st.cpu().numpy()
    ids = np.full((nq, k), -7, np.int32)
    ds = np.full((nq, k), -7.0, np.float32)
    st = np.full((nq, 3), -7, np.int32)
    lc.lc_search(h, np.ascontiguousarray(xq, np.float32), nq, sp, ids, ds, st)
    return ids, ds, st


def _clear_positions(d, nxt):
    """Positions of the oracle's returned list whose distance is clear (>= TIE relative) of
    both neighbours in the order (the one after the last being the next distance)."""
    full = np.concatenate([d, nxt[:, None]], axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.abs(np.diff(full, axis=1)) / np.maximum(np.abs(full[:, 1:]), np.abs(full[:, :-1]))
    r = np.where(np.isinf(full[:, 1:]) | np.isinf(full[:, :-1]), np.inf, r)
    clear = r >= TIE                                   # position p against p + 1
    clear[:, 1:] &= r[:, :-1] >= TIE                   # and against p - 1
    return clear


def check_valid(ref, ids, ds):
    """Every returned list is valid and every returned distance is the oracle's, recomputed
    directly for that id.  Returns nothing; asserts."""
    ctx = ref["ctx"]
    ix = ctx["ix"]
    nq, k = ids.shape
    valid = ids >= 0
    assert (ids[valid] < ix.N).all()
    # padding only at the end, with +inf
    assert (valid[:, 1:] <= valid[:, :-1]).all(), "padding before a result"
    assert np.isinf(ds[~valid]).all()
    # distinct ids per query
    srt = np.sort(np.where(valid, ids, -1 - np.arange(k)), axis=1)
    assert (np.diff(srt, axis=1) != 0).all(), "a query returned an id twice"
    # ascending by (distance, id)
    both = valid[:, 1:] & valid[:, :-1]
    up = (ds[:, 1:] > ds[:, :-1]) | ((ds[:, 1:] == ds[:, :-1]) & (ids[:, 1:] > ids[:, :-1]))
    assert up[both].all(), "a result list is out of (distance, id) order"
    walk, refined = oracle.dists(ix, ctx["Q"], np.ascontiguousarray(ids, np.int32), c1_walk=ctx["c1_walk"],
                                 walk_full=ctx["walk_full"], c2_walk=ctx["c2_walk"])
    want = walk if ctx["shortlist"] < 0 else refined
    np.testing.assert_allclose(ds[valid], want[valid], rtol=RTOL)


def _log_shares(rec):
    path = os.environ.get("LC_PARITY_LOG")
    if path:
        rec["test"] = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


def compare(ref, ids, ds, st, max_exempt=0.05, max_loss=0.002):
    """Checks one batch against the oracle (the bar in the module docstring); returns the
    share of near-tie exempt queries."""
    ok = ref["gap"] >= TIE
    walk_ok = ref["gap_walk"] >= TIE
    out_only = walk_ok & ~ok
    exempt = 1.0 - ok.mean()
    assert exempt <= max_exempt, f"{exempt:.3%} of queries are near-tie exempt"
    # decided queries: bit-exact ids and counts, distances within RTOL
    bad_ids = np.flatnonzero(ok & (ids != ref["ids"]).any(1))
    bad_st = np.flatnonzero(walk_ok & (st != ref["stats"]).any(1))
    assert bad_ids.size == 0, f"ids differ on queries {bad_ids[:10]} (of {ok.sum()} non-exempt)"
    assert bad_st.size == 0, f"visit counts differ on queries {bad_st[:10]}: {st[bad_st[:3]]} vs {ref['stats'][bad_st[:3]]}"
    fin = np.isfinite(ref["dists"][ok])
    np.testing.assert_allclose(ds[ok][fin], ref["dists"][ok][fin], rtol=RTOL)
    assert (np.isinf(ds[ok][~fin]) & (ids[ok][~fin] == -1)).all()
    # near-ties in the output order only: the same candidates, ids equal outside tie runs
    if out_only.any():
        clear = _clear_positions(ref["dists"][out_only], ref["next_dist"][out_only])
        a, b = ids[out_only], ref["ids"][out_only]
        assert np.array_equal(a[clear], b[clear]), "ids differ outside a near-tie run"
        fin = np.isfinite(ref["dists"][out_only])
        np.testing.assert_allclose(ds[out_only][fin], ref["dists"][out_only][fin], rtol=RTOL)
        assert np.array_equal(np.isinf(ds[out_only]), ~fin)
    # every query: a valid list of correctly scored ids
    check_valid(ref, ids, ds)
    # over the batch: the oracle's ids the GPU returns too
    rv = ref["ids"] >= 0
    hit = np.array([np.isin(r[m], g).sum() for r, m, g in zip(ref["ids"], rv, ids)])
    loss = 1.0 - hit.sum() / max(rv.sum(), 1)
    assert loss <= max_loss, f"the GPU misses {loss:.3%} of the oracle's ids"
    _log_shares(dict(nq=len(ids), exempt=float(exempt), walk_exempt=float(1.0 - walk_ok.mean()),
                     out_only=float(out_only.mean()), loss=float(loss)))
    return exempt


@pytest.mark.parametrize("k,ef", [(1, 16), (10, 64), (10, 256), (100, 128)])
@pytest.mark.parametrize("shortlist", [0, -1])
def test_parity_pq16(mix3k, k, ef, shortlist):
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    ref = oracle.search(ix, xq, k, ef, shortlist=shortlist)
    # every adjacent pair of the k returned is a deciding comparison: more near-ties at k = 100;
    # walks of efSearch 256 over a third of a 3,000-node graph make many deciding comparisons
    # (measured: 0.3 % at efSearch <= 64, 21 % at 256, 5 % at k = 100)
    compare(ref, *gpu_search(h, xq, k, ef, shortlist), max_exempt=0.23 if ef >= 256 else 0.07 if k >= 100 else 0.01)


@pytest.mark.parametrize("name", ["opq3k", "sift2k"])
@pytest.mark.parametrize("ef", [32, 96])
def test_parity_64_and_128_byte_codes(request, name, ef):
    ix, xb, xq = request.getfixturevalue(name)
    h = handle(name, ix)
    bound = 0.02 if ef <= 32 else 0.09                      # measured: <= 0.7 %, <= 7 %
    ref = oracle.search(ix, xq, 10, ef)
    compare(ref, *gpu_search(h, xq, 10, ef), max_exempt=bound)
    ref = oracle.search(ix, xq, 10, ef, shortlist=-1)
    compare(ref, *gpu_search(h, xq, 10, ef, shortlist=-1), max_exempt=bound)


@pytest.mark.parametrize("beam", [2, 4, 8])
@pytest.mark.parametrize("name", ["mix3k", "opq3k", "sift2k"])
def test_parity_batched(request, name, beam):
    # the batched form (beam best unexpanded members per step) against the oracle's
    ix, xb, xq = request.getfixturevalue(name)
    h = handle(name, ix)
    for shortlist in (0, -1):
        ref = oracle.search(ix, xq, 10, 64, shortlist=shortlist, beam=beam)
        compare(ref, *gpu_search(h, xq, 10, 64, shortlist, beam=beam), max_exempt=0.04)    # measured <= 3 %


def test_batched_spill_and_wide(mix3k):
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    ref = oracle.search(ix, xq, 10, 256, beam=4)
    compare(ref, *gpu_search(h, xq, 10, 256, visited_log=10, beam=4), max_exempt=0.08)    # measured 6.7 %


@pytest.mark.parametrize("tcap", [60, 250])
@pytest.mark.parametrize("beam", [1, 4])
def test_parity_tcap(opq3k, tcap, beam):
    # search-time cap T (Section 3.1): stop once T level-0 distances were computed
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    ref = oracle.search(ix, xq, 10, 128, beam=beam, tcap=tcap)
    compare(ref, *gpu_search(h, xq, 10, 128, beam=beam, tcap=tcap), max_exempt=0.01)     # measured 0


@pytest.mark.parametrize("name", ["mix3k", "opq3k", "sift2k"])
@pytest.mark.parametrize("beam", [1, 4])
def test_parity_fp16_codebook(request, name, beam):
    # FP16 form: the walk scores with C1 rounded to FP16 (nearest even); the oracle runs the
    # same definition (walk codebook rounded, FP64 arithmetic, re-rank with the FP32 C1)
    ix, xb, xq = request.getfixturevalue(name)
    h = handle(name, ix)
    c1h = ix.C1.astype(np.float16).astype(np.float32)
    for shortlist in (0, -1):
        ref = oracle.search(ix, xq, 10, 64, shortlist=shortlist, beam=beam, c1_walk=c1h)
        compare(ref, *gpu_search(h, xq, 10, 64, shortlist, beam=beam, lut_prec=lc.LC_LUT_FP16),
                max_exempt=0.035)                                                        # measured <= 2.5 %


def test_parity_10k_workload(mix10k):
    # 10k database, 1k queries, PQ16 + residual PQ16, k = 10, efSearch = 64
    ix, xb, xq = mix10k
    h = handle("mix10k", ix)
    ref = oracle.search(ix, xq, 10, 64)
    ex = compare(ref, *gpu_search(h, xq, 10, 64), max_exempt=0.025)                       # measured 1.4 %
    print(f"near-tie exempt: {ex:.2%}")


def test_host_and_device_pointers_agree_and_are_deterministic(opq3k):
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    a = gpu_search(h, xq, 10, 64, device=True)
    b = gpu_search(h, xq, 10, 64, device=False)
    c = gpu_search(h, xq, 10, 64, device=True)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_visited_spill_to_global_table(mix3k):
    # a small shared table forces the walk to continue in the per-warp global table
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    ref = oracle.search(ix, xq, 10, 256)
    assert ref["stats"][:, 0].max() > 512
    compare(ref, *gpu_search(h, xq, 10, 256, visited_log=10), max_exempt=0.23)            # measured 21 %


def test_exhaustive_walk_equals_oracle():
    # ef' >= N: every node is scored and expanded whatever the expansion order, so the
    # counts are exactly (N, N) and only the order of the returned list can hold near-ties
    from paper_1804_09996_gb300 import datagen as dg
    xt = dg.gaussian_mixture(3000, 96, 64, stream=dg.STREAM_TRAIN)
    xb = dg.gaussian_mixture(800, 96, 64, stream=dg.STREAM_BASE)
    xq = dg.gaussian_mixture(60, 96, 64, stream=dg.STREAM_QUERY)
    ix = oracle.build_index(xt, xb, 16, 16, False, codec_niter=8)
    h = handle("exh800", ix)
    k = 50
    ref = oracle.search(ix, xq, k, 1024, shortlist=-1)
    ids, ds, st = gpu_search(h, xq, k, 1024, shortlist=-1)
    assert (st[:, 0] == ix.N).all() and (st[:, 1] == ix.N).all()
    assert np.array_equal(st, ref["stats"])
    np.testing.assert_allclose(ds, ref["dists"], rtol=RTOL)
    d = oracle.search(ix, xq, k + 1, 1024, shortlist=-1)["dists"]      # one more, for the boundary
    rel = np.diff(d, axis=1) / d[:, 1:]
    # a position is decided when both of its neighbours in the order are clearly apart
    clear = np.ones_like(ids, dtype=bool)
    clear[:, 1:] &= rel[:, :k - 1] >= TIE
    clear &= rel[:, :k] >= TIE
    assert np.array_equal(ids[clear], ref["ids"][clear])
    assert clear.mean() > 0.9


def test_ragged_query_counts(mix3k):
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    for nq in (1, 3, 33, 257):
        sub = xq[:nq]
        ref = oracle.search(ix, sub, 5, 40)
        compare(ref, *gpu_search(h, sub, 5, 40), max_exempt=0.01)                          # measured <= 0.4 %


def test_empty_index_and_no_queries():
    d = 96
    import torch
    h = lc.lc_create(lc.lc_default_params(d, 16, 16))
    try:
        R = np.eye(d, dtype=np.float32)
        C = np.zeros((256, d), np.float32)
        B = np.zeros((256, 9), np.float32)
        B[:, 0] = 1
        lc.lc_import(h, 0, R, C, C, np.zeros((0, 16), np.uint8), np.zeros((0, 16), np.uint8),
                     np.zeros(0, np.uint8), B, np.zeros((0, 32), np.int32), np.zeros(0, np.int32),
                     np.zeros((0, 32), np.int32), -1)
        ids, ds, st = gpu_search(h, np.zeros((5, d), np.float32), 3, 10, device=False)
        assert (ids == -1).all() and np.isinf(ds).all() and (st == 0).all()
        ids, ds, st = gpu_search(h, np.zeros((0, d), np.float32), 3, 10, device=True)
        assert ids.shape == (0, 3)
    finally:
        lc.lc_free(h)
