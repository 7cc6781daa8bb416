"""GPU parity of the re-rank with a product regression codebook (Section 4.3: one codebook
per block of coordinates, one byte per block and vector) and with the 0-byte weights of
Section 4.2 (one least-squares weight vector per block, nothing stored per vector), against
the oracle on the same index.  Same bar as the plain parity tests."""
import numpy as np
import pytest

import oracle
from oracle.index import with_regression
from paper_1804_09996_gb300 import lc

from test_gpu_parity import compare, gpu_search

pytestmark = pytest.mark.gpu

_handles = {}


def product_index(request, name, bM, bK):
    key = (name, bM, bK)
    if key not in _handles:
        ix, xb, xq = request.getfixturevalue(name)
        ixp = with_regression(ix, bM, bK, beta_iters=4)
        h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2, beta_M=bM, beta_K=bK))
        lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ixp.beta, ixp.B, ix.adj0,
                     ix.levels, ix.upper_adj, ix.ep)
        _handles[key] = (ixp, h, xq)
    return _handles[key]


@pytest.mark.parametrize("name,bM,bK", [("opq3k", 4, 256), ("opq3k", 8, 16), ("opq3k", 1, 1),
                                        ("opq3k", 6, 1), ("mix3k", 5, 64), ("sift2k", 8, 256)])
@pytest.mark.parametrize("beam", [1, 4])
def test_parity_product_codebook(request, name, bM, bK, beam):
    ixp, h, xq = product_index(request, name, bM, bK)
    for k, shortlist in ((10, 0), (10, 32), (1, 0)):
        ref = oracle.search(ixp, xq, k, 64, shortlist=shortlist, beam=beam)
        compare(ref, *gpu_search(h, xq, k, 64, shortlist, beam=beam), max_exempt=0.06)


def test_product_codebook_changes_the_rerank(request):
    # the refined distances really depend on the per-block codewords: with every codeword
    # replaced by e0 the results are those of the plain q(x) re-rank
    ixp, h, xq = product_index(request, "opq3k", 4, 256)
    ix0 = ixp.__class__(**{**ixp.__dict__, "beta": np.zeros_like(ixp.beta)})
    a = oracle.search(ixp, xq, 10, 64)
    b = oracle.search(ix0, xq, 10, 64)
    assert not np.allclose(a["dists"], b["dists"])
    g = gpu_search(h, xq, 10, 64)
    np.testing.assert_allclose(g[1][a["gap"] >= 1e-6], a["dists"][a["gap"] >= 1e-6], rtol=1e-5)
