"""lc_search_walk_noalloc: the walk of lc_search without refinement, for callers that cannot
let the library allocate device memory while they serve (cudaMalloc/cudaFree may
synchronise the device and take unbounded time; an application that owns device memory
through its own pool or a fixed budget cannot have memory taken behind its back).  Its
scratch is a fixed array inside the library, shared by every call.

Checked through the C ABI against the existing entry point (lc_search with shortlist < 0,
the same walk) on the same index, on two calls in a row: the second call runs on the
scratch the first left behind.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1804_09996_gb300 import lc

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    import torch

    import conftest
    from paper_1804_09996_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ix, xb, xq = conftest.oracle_index("opq3k")
    h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2))
    lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0,
                 ix.levels, ix.upper_adj, ix.ep)
    yield h, ix, xq
    lc.lc_free(h)


def _outputs(nq, k):
    import torch
    return (torch.full((nq, k), -7, dtype=torch.int32, device="cuda"),
            torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda"),
            torch.full((nq, 3), -7, dtype=torch.int32, device="cuda"))


def test_not_resident_is_rejected(setup):
    import torch
    _, ix, xq = setup
    h2 = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2))
    try:
        lc.lc_import(h2, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0,
                     ix.levels, ix.upper_adj, ix.ep)
        q = torch.from_numpy(xq[:4]).cuda()
        ids, ds, st = _outputs(4, 5)
        with pytest.raises(lc.LcError) as e:
            lc.lc_search_walk_noalloc(h2, q, 4, 5, 32, ids, ds, st)
        assert e.value.status == lc.LC_ERR_STATE
    finally:
        lc.lc_free(h2)


@pytest.mark.parametrize("k,ef", [(10, 64), (1, 16), (50, 200)])
def test_matches_lc_search_on_two_calls(setup, k, ef):
    import torch
    h, ix, xq = setup
    nq = len(xq)
    q = torch.from_numpy(np.ascontiguousarray(xq)).cuda()
    s = torch.cuda.Stream()
    ref = _outputs(nq, k)
    lc.lc_search(h, q, nq, lc.lc_default_search_params(k, ef, shortlist=-1), *ref, s)   # uploads
    s.synchronize()
    ref = [t.cpu().numpy() for t in ref]
    for call in range(2):
        got = _outputs(nq, k)
        lc.lc_search_walk_noalloc(h, q, nq, k, ef, *got, s)
        s.synchronize()
        ids, ds, st = (t.cpu().numpy() for t in got)
        assert np.array_equal(ids, ref[0]), f"call {call}: ids differ"
        assert np.array_equal(st, ref[2]), f"call {call}: visit counts differ"
        fin = np.isfinite(ref[1])
        np.testing.assert_allclose(ds[fin], ref[1][fin], rtol=RTOL)
        assert np.array_equal(np.isinf(ds), ~fin)


@pytest.fixture(scope="module")
def wide():
    # 60,000 directions uniform on the sphere (no cluster structure), built by the library's
    # host build: walks at efSearch 256 score about 6,000 distinct nodes each, so every query
    # keeps most of its visited set in the global spill table
    from paper_1804_09996_gb300 import datagen as dg
    d, M1, M2 = 96, 32, 31
    h = lc.lc_create(lc.lc_default_params(d, M1, M2, use_opq=1))
    lc.lc_train(h, dg.sphere(10_000, d, stream=dg.STREAM_TRAIN))
    lc.lc_add(h, dg.sphere(60_000, d, stream=dg.STREAM_BASE))
    yield h, dg.sphere(256, d, stream=dg.STREAM_QUERY)
    lc.lc_free(h)


def test_wide_walks_match_lc_search_on_two_calls(setup, wide):
    # max(ef, k) = 256, the widest walk the call accepts, with visited sets far beyond the
    # shared-memory table: each query in flight has the spill table lc_search gives it, so
    # no query overflows and every output equals lc_search's
    import torch
    h, xq = wide
    nq, k, ef = len(xq), 10, 256
    q = torch.from_numpy(np.ascontiguousarray(xq)).cuda()
    s = torch.cuda.Stream()
    ref = _outputs(nq, k)
    lc.lc_search(h, q, nq, lc.lc_default_search_params(k, ef, shortlist=-1), *ref, s)
    s.synchronize()
    ref = [t.cpu().numpy() for t in ref]
    assert (ref[2][:, 0] > 4096).all(), "the case must visit beyond 4,096 nodes per query"
    for call in range(2):
        got = _outputs(nq, k)
        lc.lc_search_walk_noalloc(h, q, nq, k, ef, *got, s)
        s.synchronize()
        ids, ds, st = (t.cpu().numpy() for t in got)
        assert (st[:, 0] > 0).all(), f"call {call}: a query overflowed its visited tables"
        assert np.array_equal(ids, ref[0]) and np.array_equal(st, ref[2]), f"call {call}: results differ"
        np.testing.assert_allclose(ds, ref[1], rtol=RTOL)


def test_sizes_beyond_the_maximum_are_rejected(setup):
    import torch
    h, ix, xq = setup
    q = torch.from_numpy(xq[:8]).cuda()
    ids, ds, st = _outputs(8, 10)
    with pytest.raises(lc.LcError) as e:
        lc.lc_search_walk_noalloc(h, q, 8, 10, 300, ids, ds, st)
    assert e.value.status == lc.LC_ERR_ARG and "256" in e.value.message
    with pytest.raises(lc.LcError) as e:
        lc.lc_search_walk_noalloc(h, xq[:8], 8, 10, 64, ids.cpu().numpy(), ds.cpu().numpy(), None)
    assert e.value.status == lc.LC_ERR_ARG
