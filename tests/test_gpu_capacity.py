"""The visited set's capacity path: a query whose visited set outgrows its tables fails on its
own, and the batch reports it, while every other query of the batch is unaffected.

The walk keeps the visited set of Section 2's search in a shared-memory table of
2^visited_log entries, filled to three quarters, then in a global table of 2^spill_log
entries, filled to half.  Both tables are made small here (2^10 and 2^9 entries) so that, at
efSearch 192 on the 3,000-vector index, the walks that score more than 1,024 distinct nodes
(the oracle counts them) cannot fit and must fail, while those that score fewer than 962 (the
two limits less one 32-node row each, the headroom the walk keeps before a row) always fit.
Host pointers: the call returns LC_ERR_CAPACITY.  Device pointers: the failed queries
report n_dist = -1 and ids -1; every query that fits equals the oracle, as in the parity
tests.  The kernel reports the overflow and returns; nothing waits.
"""
import numpy as np
import pytest

import oracle
from paper_1804_09996_gb300 import lc
from test_gpu_parity import TIE, compare, handle

pytestmark = pytest.mark.gpu

VLOG, SLOG, EF = 10, 9, 192
SHARED = (1 << VLOG) - (1 << VLOG) // 4                # ids the shared table takes
FITS = SHARED + (1 << SLOG) // 2 - 62                  # below this, no query can fail
OVER = SHARED + (1 << SLOG) // 2                       # above this, every query must fail


def search(h, xq, k, shortlist, beam, device=True):
    import torch
    nq = len(xq)
    sp = lc.lc_default_search_params(k, EF, shortlist=shortlist, visited_log=VLOG, spill_log=SLOG)
    if beam > 1:
        sp.mode, sp.beam = lc.LC_MODE_BATCHED, beam
    if not device:
        ids = np.zeros((nq, k), np.int32)
        ds = np.zeros((nq, k), np.float32)
        lc.lc_search(h, np.ascontiguousarray(xq, np.float32), nq, sp, ids, ds, None)
        return ids, ds, None
    q = torch.from_numpy(np.ascontiguousarray(xq, np.float32)).cuda()
    ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    ds = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
    st = torch.full((nq, 3), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    lc.lc_search(h, q, nq, sp, ids, ds, st, s)
    s.synchronize()
    return ids.cpu().numpy(), ds.cpu().numpy(), st.cpu().numpy()


def rows_of(ref, rows):
    out = {key: v[rows] for key, v in ref.items() if key != "ctx"}
    out["ctx"] = dict(ref["ctx"], Q=ref["ctx"]["Q"][rows])
    return out


@pytest.mark.parametrize("shortlist", [0, -1])
@pytest.mark.parametrize("beam", [1, 4])
def test_overflowing_queries_fail_alone(mix3k, shortlist, beam):
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    ref = oracle.search(ix, xq, 10, EF, shortlist=shortlist, beam=beam)
    nd = ref["stats"][:, 0]
    decided = ref["gap_walk"] >= TIE
    must_fail = decided & (nd > OVER)
    fits = decided & (nd < FITS)
    assert must_fail.sum() >= 3 and fits.sum() >= 100
    ids, ds, st = search(h, xq, 10, shortlist, beam)
    failed = st[:, 0] == -1
    # a failed query returns nothing; a query that must fail does
    assert (ids[failed] == -1).all() and np.isinf(ds[failed]).all()
    assert failed[must_fail].all()
    assert not failed[fits].any()
    # the rest of the batch is exactly the oracle's
    ok = ~failed
    # near-tie shares of the fitting queries at efSearch 192 (from the oracle): 10.1 % plain,
    # 2.8-3.2 % batched
    compare(rows_of(ref, ok), ids[ok], ds[ok], st[ok], max_exempt=0.13)
    # host pointers: the batch reports the overflow
    with pytest.raises(lc.LcError) as e:
        search(h, xq, 10, shortlist, beam, device=False)
    assert e.value.status == lc.LC_ERR_CAPACITY


def test_queries_that_fit_report_no_overflow(mix3k):
    # the same small tables, only queries that fit: the host-pointer call succeeds
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    ref = oracle.search(ix, xq, 10, EF)
    small = np.flatnonzero(ref["stats"][:, 0] < FITS - 100)[:64]
    assert len(small) >= 32
    ids, ds, _ = search(h, xq[small], 10, 0, 1, device=False)
    assert (ids >= 0).all()
