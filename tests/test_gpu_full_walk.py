"""GPU parity of the walk on the full two-level decode q = c1 + c2 (lc_search_params.walk_full;
Section 4.1's approximation taken in full, instead of the level-1 code alone) against the
oracle's full walk on the same index, for the three uniform level-1 splits (16 and 32
sub-spaces at d = 96, 64 at d = 128), plain and batched, FP32 and FP16 codebooks (the oracle
decodes with the same rounded codebooks).  Same bar as the other parity tests."""
import numpy as np
import pytest

import oracle
from paper_1804_09996_gb300 import lc

from test_gpu_parity import compare, gpu_search, handle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["mix3k", "opq3k", "sift2k"])
@pytest.mark.parametrize("beam", [1, 4])
@pytest.mark.parametrize("prec", [lc.LC_LUT_FP32, lc.LC_LUT_FP16])
def test_parity_full_walk(request, name, beam, prec):
    ix, xb, xq = request.getfixturevalue(name)
    h = handle(name, ix)
    kw = {}
    if prec == lc.LC_LUT_FP16:
        kw = dict(c1_walk=ix.C1.astype(np.float16).astype(np.float32),
                  c2_walk=ix.C2.astype(np.float16).astype(np.float32))
    for shortlist in (0, -1):
        ref = oracle.search(ix, xq, 10, 64, shortlist=shortlist, beam=beam, walk_full=True, **kw)
        got = gpu_search(h, xq, 10, 64, shortlist, beam=beam, lut_prec=prec, walk_full=1)
        compare(ref, *got, max_exempt=0.04)


@pytest.mark.parametrize("beam", [1, 4])
def test_parity_full_walk_uneven_split(odd2k, beam):
    # FP32 full walk with non-uniform level-1 and level-2 splits (d = 40, M1 = 16, M2 = 10)
    ix, xb, xq = odd2k
    h = handle("odd2k", ix)
    for shortlist in (0, -1):
        ref = oracle.search(ix, xq, 10, 48, shortlist=shortlist, beam=beam, walk_full=True)
        compare(ref, *gpu_search(h, xq, 10, 48, shortlist, beam=beam, walk_full=1), max_exempt=0.04)
        ref = oracle.search(ix, xq, 10, 48, shortlist=shortlist, beam=beam)
        compare(ref, *gpu_search(h, xq, 10, 48, shortlist, beam=beam), max_exempt=0.04)


def test_full_walk_differs_from_level1_walk(opq3k):
    # the two walks score different things: their visit counts differ on most queries
    ix, xb, xq = opq3k
    h = handle("opq3k", ix)
    a = gpu_search(h, xq, 10, 64, -1)
    b = gpu_search(h, xq, 10, 64, -1, walk_full=1)
    assert (a[2][:, 0] != b[2][:, 0]).mean() > 0.5


def test_full_walk_fp16_needs_uniform_split():
    d, M1, M2, n = 40, 16, 8, 300
    rng = np.random.default_rng(3)
    h = lc.lc_create(lc.lc_default_params(d, M1, M2, use_opq=0, kmeans_iters=3, beta_iters=1))
    try:
        lc.lc_train(h, rng.standard_normal((600, d)).astype(np.float32))
        lc.lc_add(h, rng.standard_normal((n, d)).astype(np.float32))
        q = rng.standard_normal((4, d)).astype(np.float32)
        ids = np.empty((4, 10), np.int32)
        ds = np.empty((4, 10), np.float32)
        lc.lc_search(h, q, 4, lc.lc_default_search_params(10, 32), ids, ds)
        lc.lc_search(h, q, 4, lc.lc_default_search_params(10, 32, walk_full=1), ids, ds)
        with pytest.raises(lc.LcError) as e:
            lc.lc_search(h, q, 4, lc.lc_default_search_params(10, 32, walk_full=1, lut_prec=lc.LC_LUT_FP16), ids, ds)
        assert e.value.status == lc.LC_ERR_ARG and "uniform" in e.value.message
    finally:
        lc.lc_free(h)
