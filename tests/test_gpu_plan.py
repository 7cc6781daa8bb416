"""Captured search plans (lc_plan_*): the whole search recorded once into a CUDA graph over
buffers the plan owns.  Every run must return exactly what lc_search(_ex) returns for the
same queries and parameters, for any batch size up to the plan's largest (sizes changing
from run to run update the graph's kernel nodes), for uint8 queries and per-query
efSearch; a plan refuses to run once its index has changed."""
import numpy as np
import pytest

from paper_1804_09996_gb300 import datagen, lc

from test_gpu_parity import gpu_search, handle
from test_gpu_uneven import search_ex

pytestmark = pytest.mark.gpu


def _plan_search(pl, t, q, efq=None, stream=None):
    import torch
    n = len(q)
    t["q"][:n].copy_(torch.from_numpy(np.ascontiguousarray(q)))
    if efq is not None:
        t["ef"][:n].copy_(torch.from_numpy(np.ascontiguousarray(efq, np.int32)))
    torch.cuda.synchronize()
    lc.lc_plan_run(pl, n, stream)
    torch.cuda.synchronize()
    return t["ids"][:n].cpu().numpy(), t["dists"][:n].cpu().numpy(), t["stats"][:n].cpu().numpy()


@pytest.mark.parametrize("beam,shortlist", [(1, 0), (4, 0), (1, -1), (8, 20)])
def test_plan_equals_search_for_changing_sizes(opq3k, beam, shortlist):
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    sp = lc.lc_default_search_params(10, 64, shortlist=shortlist)
    if beam > 1:
        sp.mode, sp.beam = lc.LC_MODE_BATCHED, beam
    pl = lc.lc_plan_create(h, 256, sp)
    try:
        t = lc.lc_plan_tensors(pl, 256, ix.d, 10)
        for n in (256, 1, 100, 0, 37, 256, 37):
            got = _plan_search(pl, t, xq[:n])
            ref = gpu_search(h, xq[:n], 10, 64, shortlist, beam=beam) if n else None
            for a, b in zip(got, ref or [np.empty((0, 10)), np.empty((0, 10)), np.empty((0, 3))]):
                assert np.array_equal(a, b), n
    finally:
        lc.lc_plan_free(pl)


def test_plan_u8_and_per_query_ef(sift2k):
    ix, xb, xq = sift2k
    h = handle("sift2k", ix)
    sp = lc.lc_default_search_params(10, 256)
    pl = lc.lc_plan_create(h, len(xq), sp, lc.LC_QUERY_U8, True)
    try:
        t = lc.lc_plan_tensors(pl, len(xq), ix.d, 10, lc.LC_QUERY_U8)
        efq = datagen.uneven_ef(len(xq))
        for n in (len(xq), 50):
            got = _plan_search(pl, t, xq[:n].astype(np.uint8), efq[:n])
            ref = search_ex(h, xq[:n].astype(np.uint8), 10, 256, efq[:n], u8=True)
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
    finally:
        lc.lc_plan_free(pl)


def test_plan_refuses_a_changed_index(mix3k):
    ix, xb, xq = mix3k
    h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2))
    args = (ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0, ix.levels, ix.upper_adj, ix.ep)
    lc.lc_import(h, *args)
    pl = lc.lc_plan_create(h, 16, lc.lc_default_search_params(10, 32))
    try:
        lc.lc_plan_run(pl, 16)
        with pytest.raises(lc.LcError) as e:
            lc.lc_plan_run(pl, 17)
        assert e.value.status == lc.LC_ERR_ARG
        lc.lc_import(h, *args)
        with pytest.raises(lc.LcError) as e:
            lc.lc_plan_run(pl, 16)
        assert e.value.status == lc.LC_ERR_STATE
    finally:
        lc.lc_plan_free(pl)
        lc.lc_free(h)
