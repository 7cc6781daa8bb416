"""Ordered search (lc_search_params.order): the upper-level descents run as their own launch,
the queries are sorted by decreasing distance to their level-0 entry node, and the level-0
walks run in that order.  Each query's computation is unchanged, so ordered and query-order
results must be identical bit for bit (ids, distances, visit counts) for every form of the
search, and both must match the oracle."""
import numpy as np
import pytest

import oracle
from paper_1804_09996_gb300 import lc
from test_gpu_parity import compare, handle
from test_gpu_uneven import oracle_uneven

pytestmark = pytest.mark.gpu


def search(h, xq, k, ef, order, beam=1, lut_prec=0, tcap=0, walk_full=0, efq=None, u8=False, shortlist=0):
    import torch
    nq = len(xq)
    sp = lc.lc_default_search_params(k, ef, shortlist=shortlist, lut_prec=lut_prec, max_dist=tcap,
                                     walk_full=walk_full, order=order)
    if beam > 1:
        sp.mode, sp.beam = lc.LC_MODE_BATCHED, beam
    q = torch.from_numpy(np.ascontiguousarray(xq, np.uint8 if u8 else np.float32)).cuda()
    e = None if efq is None else torch.from_numpy(np.ascontiguousarray(efq, np.int32)).cuda()
    ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    ds = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
    st = torch.full((nq, 3), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    lc.lc_search_ex(h, q, lc.LC_QUERY_U8 if u8 else lc.LC_QUERY_F32, nq, sp, e, ids, ds, st, s)
    s.synchronize()
    return ids.cpu().numpy(), ds.cpu().numpy(), st.cpu().numpy()


def same(a, b):
    assert np.array_equal(a[0], b[0]), "ids differ between ordered and query-order walks"
    assert np.array_equal(a[1].view(np.int32), b[1].view(np.int32)), "distances differ"
    assert np.array_equal(a[2], b[2]), "visit counts differ"


FORMS = [dict(), dict(beam=4), dict(lut_prec=lc.LC_LUT_FP16), dict(beam=4, lut_prec=lc.LC_LUT_FP16),
         dict(tcap=200), dict(shortlist=-1, beam=2)]


@pytest.mark.parametrize("form", range(len(FORMS)))
@pytest.mark.parametrize("name", ["mix3k", "opq3k"])
def test_ordered_equals_query_order_and_oracle(request, name, form):
    ix, xb, xq = request.getfixturevalue(name)
    h = handle(name, ix)
    f = FORMS[form]
    a = search(h, xq, 10, 64, lc.LC_ORDER_ALWAYS, **f)
    b = search(h, xq, 10, 64, lc.LC_ORDER_NEVER, **f)
    same(a, b)
    c1h = ix.C1.astype(np.float16).astype(np.float32) if f.get("lut_prec") else None
    ref = oracle.search(ix, xq, 10, 64, shortlist=f.get("shortlist", 0), beam=f.get("beam", 1),
                        tcap=f.get("tcap", 0), c1_walk=c1h)
    compare(ref, *a, max_exempt=0.06)                     # measured <= 4.7 %


def test_ordered_uint8_per_query_ef(sift2k):
    from paper_1804_09996_gb300 import datagen
    ix, xb, xq = sift2k
    h = handle("sift2k", ix)
    efq = datagen.uneven_ef(len(xq), choices=(16, 32, 64, 128))
    q8 = np.clip(np.rint(xq), 0, 255).astype(np.uint8)
    a = search(h, q8, 10, 128, lc.LC_ORDER_ALWAYS, efq=efq, u8=True, beam=4)
    b = search(h, q8, 10, 128, lc.LC_ORDER_NEVER, efq=efq, u8=True, beam=4)
    same(a, b)
    ref = oracle_uneven(ix, q8.astype(np.float32), 10, efq, beam=4)
    compare(ref, *a, max_exempt=0.02)                     # measured 0


def test_ordered_full_walk(opq3k):
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    a = search(h, xq, 10, 32, lc.LC_ORDER_ALWAYS, walk_full=1, beam=4)
    b = search(h, xq, 10, 32, lc.LC_ORDER_NEVER, walk_full=1, beam=4)
    same(a, b)


def test_ordered_single_query_and_auto(mix3k):
    # one query (the sort of one key), and the automatic choice on a small batch (query order)
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    for n in (1, 33):
        a = search(h, xq[:n], 10, 64, lc.LC_ORDER_ALWAYS)
        b = search(h, xq[:n], 10, 64, lc.LC_ORDER_AUTO)
        same(a, b)
