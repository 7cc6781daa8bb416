"""Serving (lc_serve_*): requests of mixed size, k, efSearch and mode admitted by a device
memory budget; requests of the same parameters that wait while the launch slots are busy run
merged into one launch, each query with its own request's efSearch.  Each request's results
must be exactly what lc_search returns for it alone, and (served mix with efSearch up to 512)
the oracle's; a request that can never fit the budget is rejected at submission; queued
requests wait for room and are cancelled at close."""
import numpy as np
import pytest

from paper_1804_09996_gb300 import lc


def test_serve_open_errors_without_gpu():
    h = lc.lc_create(lc.lc_default_params(16, 16, 8, use_opq=0))
    try:
        with pytest.raises(lc.LcError) as e:
            lc.lc_serve_open(h, 1 << 30, 4, 64)
        assert e.value.status == lc.LC_ERR_STATE
        with pytest.raises(lc.LcError) as e:
            lc.lc_serve_open(h, 1 << 30, 0, 64)
        assert e.value.status == lc.LC_ERR_ARG
    finally:
        lc.lc_free(h)


def _requests(rng, xq, n):
    """n requests: sizes log-uniform in [1, 64], k in {1, 10, 100}, efSearch log-uniform in
    [16, 512], plain or batched."""
    out = []
    for _ in range(n):
        size = int(np.exp(rng.uniform(0, np.log(64))))
        start = int(rng.integers(0, len(xq) - size))
        k = int(rng.choice([1, 10, 100]))
        ef = int(np.exp(rng.uniform(np.log(16), np.log(512))))
        sp = lc.lc_default_search_params(k, ef)
        if rng.random() < 0.5:
            sp.mode, sp.beam = lc.LC_MODE_BATCHED, int(rng.choice([2, 4]))
        out.append((xq[start:start + size], sp))
    return out


def _alone(h, q, sp):
    ids = np.empty((len(q), sp.k), np.int32)
    ds = np.empty((len(q), sp.k), np.float32)
    lc.lc_search(h, np.ascontiguousarray(q), len(q), sp, ids, ds)
    return ids, ds


def _run(srv, reqs, poll_ms=50):
    results, cbs, ids = {}, [], []
    for q, sp in reqs:
        cb = lc.make_request_cb(lambda rid, st, i, d: results.__setitem__(rid, (st, i, d)))
        cbs.append(cb)
        ids.append(lc.lc_serve_submit(srv, q, sp, cb))
    for _ in range(100000):
        if len(results) == len(reqs):
            break
        lc.lc_serve_poll(srv, poll_ms)
    return ids, results, cbs


@pytest.fixture(scope="module")
def served():
    import conftest
    from paper_1804_09996_gb300 import build
    build.build()
    ix, xb, xq = conftest.oracle_index("opq3k")
    h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2))
    lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0,
                 ix.levels, ix.upper_adj, ix.ep)
    yield h, xq, ix
    lc.lc_free(h)


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix(served, rng):
    h, xq, ix = served
    reqs = _requests(rng, xq, 60)
    srv = lc.lc_serve_open(h, 4 << 30, 16, 64)
    try:
        ids, results, _ = _run(srv, reqs)
    finally:
        lc.lc_serve_close(srv)
    assert len(results) == len(reqs)
    for rid, (q, sp) in zip(ids, reqs):
        st, i, d = results[rid]
        assert st == lc.LC_OK
        ai, ad = _alone(h, q, sp)
        assert np.array_equal(i, ai)
        assert np.array_equal(d, ad)


@pytest.mark.gpu
def test_budget_admission_and_rejection(served, rng):
    h, xq, ix = served
    sp = lc.lc_default_search_params(10, 64)
    tiny = lc.lc_serve_open(h, 64 << 10, 4, 64)
    try:
        with pytest.raises(lc.LcError) as e:
            lc.lc_serve_submit(tiny, xq[:8], sp, lc.make_request_cb(lambda *a: None))
        assert e.value.status == lc.LC_ERR_BUDGET
        with pytest.raises(lc.LcError) as e:
            lc.lc_serve_submit(tiny, xq[:65], sp, lc.make_request_cb(lambda *a: None))
        assert e.value.status == lc.LC_ERR_BUDGET
    finally:
        lc.lc_serve_close(tiny)
    # a budget that holds one such request at a time (~0.7 MB of state, mostly the visited
    # spill tables of its warps): the others wait in order, all complete
    reqs = [(xq[i * 16:(i + 1) * 16], sp) for i in range(5)]
    one = lc.lc_serve_open(h, 1 << 20, 4, 64)
    try:
        ids, results, _ = _run(one, reqs)
    finally:
        lc.lc_serve_close(one)
    assert sorted(results) == sorted(ids)
    for rid, (q, s2) in zip(ids, reqs):
        st, i, d = results[rid]
        assert st == lc.LC_OK
        assert np.array_equal(i, _alone(h, q, s2)[0])


@pytest.mark.gpu
def test_close_cancels_requests_not_started(served):
    h, xq, ix = served
    sp = lc.lc_default_search_params(10, 64)
    srv = lc.lc_serve_open(h, 1 << 30, 1, 64)
    seen = {}
    cbs = [lc.make_request_cb(lambda rid, st, i, d: seen.__setitem__(rid, st)) for _ in range(4)]
    ids = [lc.lc_serve_submit(srv, xq[j * 8:(j + 1) * 8], sp, cbs[j]) for j in range(4)]
    lc.lc_serve_close(srv)
    assert seen[ids[0]] == lc.LC_OK                  # already on the device: completes
    assert all(seen[r] == lc.LC_ERR_STATE for r in ids[1:])


@pytest.mark.gpu
def test_waiting_requests_run_merged_and_equal_alone(served):
    # one launch slot: the first request runs alone, the 23 that queue behind it share its
    # parameters (efSearch 33..64, one class) and run as one merged launch once it is done
    h, xq, ix = served
    rng = np.random.default_rng(3)
    reqs = []
    for j in range(24):
        size = int(rng.integers(1, 40))
        s0 = int(rng.integers(0, len(xq) - size))
        reqs.append((xq[s0:s0 + size], lc.lc_default_search_params(10, int(rng.integers(33, 65)))))
    srv = lc.lc_serve_open(h, 1 << 30, 1, 64)
    try:
        ids, results, _ = _run(srv, reqs)
    finally:
        lc.lc_serve_close(srv)
    for rid, (q, sp) in zip(ids, reqs):
        st, i, d = results[rid]
        assert st == lc.LC_OK
        ai, ad = _alone(h, q, sp)
        assert np.array_equal(i, ai) and np.array_equal(d, ad)


@pytest.mark.gpu
def test_served_mix_against_the_oracle(served):
    # a served mix (k 1 or 10, efSearch 16..512, FP32 and FP16 codebooks, two launch slots so
    # that requests queue and merge) checked request by request against the oracle with the
    # parity bar of the batch search (the server does not return visit counts; those are
    # checked by the batch parity tests)
    import oracle
    from test_gpu_parity import compare
    h, xq, ix = served
    rng = np.random.default_rng(11)
    c1h = ix.C1.astype(np.float16).astype(np.float32)
    reqs = []
    for j in range(40):
        size = int(rng.integers(4, 48))
        s0 = int(rng.integers(0, len(xq) - size))
        ef = int(np.exp(rng.uniform(np.log(16), np.log(512))))
        if j < 4:
            ef = 512
        sp = lc.lc_default_search_params(int(rng.choice([1, 10])), ef, lut_prec=int(j % 2))
        reqs.append((xq[s0:s0 + size], sp))
    srv = lc.lc_serve_open(h, 1 << 30, 2, 64)
    try:
        ids, results, _ = _run(srv, reqs)
    finally:
        lc.lc_serve_close(srv)
    # each request against the oracle at its own efSearch, checked together per (k, codebook)
    groups = {}
    for rid, (q, sp) in zip(ids, reqs):
        st, i, d = results[rid]
        assert st == lc.LC_OK
        ref = oracle.search(ix, q, sp.k, sp.ef, c1_walk=c1h if sp.lut_prec else None)
        groups.setdefault((sp.k, sp.lut_prec), []).append((q, i, d, ref))
    for (k, prec), rows in groups.items():
        ref = {key: np.concatenate([r[3][key] for r in rows]) for key in
               ("ids", "dists", "stats", "gap", "gap_walk", "next_dist")}
        ref["ctx"] = dict(rows[0][3]["ctx"], Q=np.ascontiguousarray(np.concatenate([r[0] for r in rows]), np.float32))
        i = np.concatenate([r[1] for r in rows])
        d = np.concatenate([r[2] for r in rows])
        # walks of efSearch up to 512 on a 3,000-vector index make many deciding comparisons
        compare(ref, i, d, ref["stats"], max_exempt=0.35, max_loss=0.01)
