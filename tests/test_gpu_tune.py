"""Autotuner (lc_autotune): the parameters it returns reach the plain search's 1-recall@1 on
the sample, the recall and the parameters it reports are what lc_search then gives, and its
launch-shape stage leaves results unchanged."""
import numpy as np
import pytest

import oracle
from paper_1804_09996_gb300 import lc

from test_gpu_parity import gpu_search, handle

pytestmark = pytest.mark.gpu


def _search(h, q, sp):
    ids = np.empty((len(q), sp.k), np.int32)
    ds = np.empty((len(q), sp.k), np.float32)
    lc.lc_search(h, np.ascontiguousarray(q, np.float32), len(q), sp, ids, ds)
    return ids, ds


@pytest.mark.parametrize("with_gt,batch", [(True, 0), (False, 0), (True, 4000)])
def test_autotune_meets_target(mix10k, with_gt, batch):
    ix, xb, xq = mix10k
    h = handle("mix10k", ix)
    gt = oracle.knn(xb, xq, 1)[0][:, 0].astype(np.int32) if with_gt else None
    r = lc.lc_autotune(h, xq, gt, k=10, ef=48, reps=2, batch=batch)
    assert r.tried > 10
    assert r.recall >= r.target > 0.3
    assert r.ms <= r.base_ms
    ids, _ = _search(h, xq, r.sp)
    ref = gt if with_gt else _search(h, xq, lc.lc_default_search_params(10, 192))[0][:, 0]
    assert abs((ids[:, 0] == ref).mean() - r.recall) < 1e-6
    # the launch shape (warps per block, visited table) never changes results
    sp0 = lc.lc_search_params.from_buffer_copy(r.sp)
    sp0.warps, sp0.visited_log = 0, 0
    ids0, ds0 = _search(h, xq, sp0)
    got = _search(h, xq, r.sp)
    assert np.array_equal(ids0, got[0]) and np.array_equal(ds0, got[1])


@pytest.mark.parametrize("warps", [1, 3, 8, 16])
@pytest.mark.parametrize("vlog", [10, 13])
def test_launch_shape_does_not_change_results(opq3k, warps, vlog):
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    ref = gpu_search(h, xq, 10, 96, beam=4)
    sp = lc.lc_default_search_params(10, 96, mode=lc.LC_MODE_BATCHED, beam=4, warps=warps, visited_log=vlog)
    ids, ds = _search(h, xq, sp)
    assert np.array_equal(ids, ref[0]) and np.array_equal(ds, ref[1])
