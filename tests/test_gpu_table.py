"""The table form (LC_LUT_TABLE): Section 4.1's per-query ADC tables built on the tensor cores.

A kernel builds, for the whole batch, every query's table of ||y'_j - C1_j[c]||^2 over the 32
level-1 sub-spaces and 256 centroids (y' and C1 rounded to FP16, FP16 tensor-core products with
FP32 accumulation, entries stored in FP16), and the walk adds table entries instead of
computing terms from the codebook.  The distances change at FP16 precision, so this form is
checked as a precision form: every returned distance against the unrounded FP64 ADC distance
of the same id (the oracle's definition), the result lists for validity, recall against the
exact nearest neighbours compared with the FP32 form, and determinism.
"""
import numpy as np
import pytest

import oracle
from paper_1804_09996_gb300 import lc
from test_gpu_parity import gpu_search, handle

pytestmark = pytest.mark.gpu


def check_list(ids, ds, N):
    valid = ids >= 0
    assert (ids[valid] < N).all()
    assert (valid[:, 1:] <= valid[:, :-1]).all()
    both = valid[:, 1:] & valid[:, :-1]
    up = (ds[:, 1:] > ds[:, :-1]) | ((ds[:, 1:] == ds[:, :-1]) & (ids[:, 1:] > ids[:, :-1]))
    assert up[both].all()
    for row, v in zip(ids, valid):
        assert len(set(row[v].tolist())) == v.sum()


@pytest.mark.parametrize("beam", [1, 4])
def test_table_distances_against_the_unrounded_oracle(opq3k, beam):
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    ids, ds, st = gpu_search(h, xq, 10, 64, shortlist=-1, beam=beam, lut_prec=lc.LC_LUT_TABLE)
    check_list(ids, ds, ix.N)
    exact, _ = oracle.dists(ix, xq, ids)
    v = ids >= 0
    rel = np.abs(ds[v].astype(np.float64) - exact[v]) / exact[v]
    q = np.percentile(rel, [50, 99, 100])
    print(f"table form (beam {beam}): ADC distance vs the unrounded FP64 oracle: median {q[0]:.2e}, "
          f"p99 {q[1]:.2e}, max {q[2]:.2e} relative")
    assert q[0] < 2e-3 and q[2] < 3e-2


def test_table_recall_matches_the_fp32_form(opq3k):
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    gt, _ = oracle.knn(xb, xq, 1)
    r = {}
    for name, prec in (("fp32", lc.LC_LUT_FP32), ("table", lc.LC_LUT_TABLE)):
        ids = gpu_search(h, xq, 10, 64, beam=4, lut_prec=prec)[0]
        r[name] = float((ids[:, 0] == gt[:, 0]).mean())
    print(f"R@1 fp32 {r['fp32']:.4f}, table {r['table']:.4f}")
    assert r["table"] > 0.5 and abs(r["table"] - r["fp32"]) <= 0.02


def test_table_form_is_deterministic_and_device_host_agree(opq3k):
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    a = gpu_search(h, xq, 10, 64, beam=4, lut_prec=lc.LC_LUT_TABLE)
    b = gpu_search(h, xq, 10, 64, beam=4, lut_prec=lc.LC_LUT_TABLE, device=False)
    c = gpu_search(h, xq, 10, 64, beam=4, lut_prec=lc.LC_LUT_TABLE)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_table_form_rejected_where_it_is_not_built(mix3k, opq3k):
    # 16 sub-spaces of 6 coordinates: not the table kernel's shape
    ix, xb, xq = mix3k
    h = handle("mix3k", ix)
    with pytest.raises(lc.LcError) as e:
        gpu_search(h, xq[:4], 10, 64, lut_prec=lc.LC_LUT_TABLE)
    assert e.value.status == lc.LC_ERR_ARG
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    with pytest.raises(lc.LcError) as e:
        gpu_search(h, xq[:4], 10, 64, lut_prec=lc.LC_LUT_TABLE, walk_full=1)
    assert e.value.status == lc.LC_ERR_ARG


def test_table_form_ordered_equals_query_order(opq3k):
    # the descent launch of an ordered search scores with the same tables as the walk
    from test_gpu_order import same, search
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    for f in (dict(), dict(beam=4), dict(beam=2, shortlist=-1)):
        a = search(h, xq, 10, 64, lc.LC_ORDER_ALWAYS, lut_prec=lc.LC_LUT_TABLE, **f)
        b = search(h, xq, 10, 64, lc.LC_ORDER_NEVER, lut_prec=lc.LC_LUT_TABLE, **f)
        same(a, b)


def test_table_form_plan_equals_search(opq3k):
    from test_gpu_plan import _plan_search
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    sp = lc.lc_default_search_params(10, 64, lut_prec=lc.LC_LUT_TABLE)
    sp.mode, sp.beam = lc.LC_MODE_BATCHED, 4
    pl = lc.lc_plan_create(h, 256, sp)
    try:
        t = lc.lc_plan_tensors(pl, 256, ix.d, 10)
        for n in (256, 1, 37, 256):
            got = _plan_search(pl, t, xq[:n])
            ref = gpu_search(h, xq[:n], 10, 64, beam=4, lut_prec=lc.LC_LUT_TABLE)
            for x, y in zip(got, ref):
                assert np.array_equal(x, y), n
    finally:
        lc.lc_plan_free(pl)


def test_table_form_served_equals_alone(opq3k, rng):
    from test_serve import _alone, _run
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    reqs = []
    for _ in range(24):
        size = int(rng.integers(1, 48))
        start = int(rng.integers(0, len(xq) - size))
        sp = lc.lc_default_search_params(int(rng.choice([1, 10])), int(rng.choice([32, 64, 128])),
                                         lut_prec=lc.LC_LUT_TABLE)
        if rng.random() < 0.5:
            sp.mode, sp.beam = lc.LC_MODE_BATCHED, 4
        reqs.append((xq[start:start + size], sp))
    srv = lc.lc_serve_open(h, 1 << 30, 2, 64)
    try:
        ids, results, _ = _run(srv, reqs)
    finally:
        lc.lc_serve_close(srv)
    assert len(results) == len(reqs)
    for rid, (q, sp) in zip(ids, reqs):
        st, i, d = results[rid]
        assert st == lc.LC_OK
        ai, ad = _alone(h, q, sp)
        assert np.array_equal(i, ai) and np.array_equal(d, ad)
