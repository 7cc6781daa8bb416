"""The library's host build (lc_train / lc_add) checked on the CPU against the oracle and
against properties the paper fixes: PQ codes are the brute-force argmin under the
library's own codebooks, the OPQ rotation is orthogonal, the graph has HNSW's structure,
codeword 0 is e0 and every vector's codeword minimises its refinement loss, and searching
the library-built index (with the oracle) finds neighbours as well as the oracle's own
build does."""
import numpy as np
import pytest

import oracle
from oracle import codec, refine
from oracle.graph import upper_offsets
from oracle.index import OracleIndex
from paper_1804_09996_gb300 import datagen as dg
from paper_1804_09996_gb300 import lc
from test_oracle_graph import check_structure


@pytest.fixture(scope="module")
def libbuilt():
    from paper_1804_09996_gb300 import build
    build.build()
    d, M1, M2 = 96, 32, 31
    xt = dg.gaussian_mixture(6000, d, 256, stream=dg.STREAM_TRAIN)
    xb = dg.gaussian_mixture(4000, d, 256, stream=dg.STREAM_BASE)
    xq = dg.gaussian_mixture(300, d, 256, stream=dg.STREAM_QUERY)
    h = lc.lc_create(lc.lc_default_params(d, M1, M2, use_opq=1, opq_iters=4, kmeans_iters=10,
                                          batch_max=256))
    lc.lc_train(h, xt)
    lc.lc_add(h, xb)
    ex = lc.lc_export(h, d, M1, M2)
    lc.lc_free(h)
    off, _ = upper_offsets(ex["levels"])
    ix = OracleIndex(d=d, M1=M1, M2=M2, R=ex["R"], C1=ex["C1"], C2=ex["C2"], codes1=ex["codes1"],
                     codes2=ex["codes2"], beta=ex["beta"], B=ex["B"], adj0=ex["adj0"], upper_off=off,
                     upper_adj=ex["upper_adj"], ep=ex["ep"], max_level=int(ex["levels"].max()),
                     levels=ex["levels"])
    xr = xb.astype(np.float64) @ ix.R.astype(np.float64).T
    ix.extra.update(xr=xr, xh=ix.decoded())
    return ix, xt, xb, xq


def test_rotation_orthogonal(libbuilt):
    ix = libbuilt[0]
    R = ix.R.astype(np.float64)
    assert np.abs(R @ R.T - np.eye(ix.d)).max() < 1e-5


def test_codes_are_argmin_under_library_codebooks(libbuilt):
    ix, _, xb, _ = libbuilt
    xr = ix.extra["xr"][:500]
    c1 = codec.pq_encode(xr, ix.C1.astype(np.float64), ix.M1)
    agree1 = (c1 == ix.codes1[:500]).mean()
    res = xr - codec.pq_decode(ix.codes1[:500], ix.C1.astype(np.float64), ix.M1)
    c2 = codec.pq_encode(res, ix.C2.astype(np.float64), ix.M2)
    agree2 = (c2 == ix.codes2[:500]).mean()
    # FP32 (library) vs FP64 (oracle) argmin may only differ on near-ties
    assert agree1 > 0.999 and agree2 > 0.999, (agree1, agree2)


def test_graph_structure(libbuilt):
    check_structure(libbuilt[0])


def test_graph_equals_the_oracle_build_on_the_same_codes(libbuilt):
    # Section 5.1's batched insertion, restated by the oracle in FP64 (orc_build_graph) on the
    # library's own rotation, codes and levels: the library's host build gives the same graph,
    # row for row and in row order, at level 0 and above, with the same entry point
    from oracle.graph import build_graph
    ix = libbuilt[0]
    a0, off, ua, ep, ml = build_graph(ix.extra["xr"], ix.extra["xh"], ix.levels, deg=32, deg_up=32, efc=40,
                                      batch_max=256, batch_div=16)
    assert np.array_equal(a0, ix.adj0)
    assert np.array_equal(ua, ix.upper_adj) and np.array_equal(off, ix.upper_off)
    assert ep == ix.ep and ml == ix.max_level


def test_codewords_minimise_refinement_loss(libbuilt):
    ix = libbuilt[0]
    assert np.array_equal(ix.B[0], refine.e0().astype(np.float32))
    xh, xr = ix.extra["xh"], ix.extra["xr"]
    idx = np.arange(800)
    G = refine.gmatrix(xh, ix.adj0, idx)
    best = refine.assign_codewords(G, xr[idx], ix.B.astype(np.float64))
    L = refine.losses(G, xr[idx], ix.B.astype(np.float64))
    got = L[np.arange(len(idx)), ix.beta[idx].astype(np.int64)]
    # the library's choice is the oracle's argmin, or ties with it to rounding
    assert np.all(got <= L[np.arange(len(idx)), best] * (1 + 1e-5) + 1e-9)
    assert (best == ix.beta[idx]).mean() > 0.98
    base = ((xr - xh) ** 2).sum(1)
    refined = refine.losses_assigned(refine.gmatrix(xh, ix.adj0, np.arange(ix.N)), xr, ix.B.astype(np.float64),
                                     ix.beta.astype(np.int64))
    assert np.all(refined <= base * (1 + 1e-5) + 1e-9)


def test_library_index_searches_as_well_as_oracle_build(libbuilt):
    ix, xt, xb, xq = libbuilt
    gt, _ = oracle.knn(xb, xq, 1)
    r_lib = oracle.search(ix, xq, k=10, ef=64)
    oix = oracle.build_index(xt, xb, 32, 31, True, opq_outer=4, codec_niter=10, batch_max=256)
    r_orc = oracle.search(oix, xq, k=10, ef=64)
    rl = (r_lib["ids"][:, 0] == gt[:, 0]).mean()
    ro = (r_orc["ids"][:, 0] == gt[:, 0]).mean()
    assert rl > 0.6 and abs(rl - ro) < 0.08, (rl, ro)


def test_add_in_two_calls_keeps_ids_and_structure():
    d = 32
    xt = dg.gaussian_mixture(2000, d, 32, stream=dg.STREAM_TRAIN)
    xb = dg.gaussian_mixture(1500, d, 32, stream=dg.STREAM_BASE)
    h = lc.lc_create(lc.lc_default_params(d, 16, 8, use_opq=0, kmeans_iters=5))
    try:
        lc.lc_train(h, xt)
        lc.lc_add(h, xb[:700])
        lc.lc_add(h, xb[700:])
        assert lc.lc_size(h) == 1500
        ex = lc.lc_export(h, d, 16, 8)
        ref = codec.pq_encode(xb.astype(np.float64), ex["C1"].astype(np.float64), 16)
        assert (ref == ex["codes1"]).mean() > 0.999
        adj = ex["adj0"]
        assert ((adj >= -1) & (adj < 1500)).all()
        assert (adj[700:] >= 0).sum(1).min() >= 1
    finally:
        lc.lc_free(h)


def test_build_does_not_depend_on_the_thread_count():
    # every parallel reduction of train/add has a fixed order: 1, 3 and all threads build the
    # same index bit for bit (OPQ rotation, both codebooks, codes, graph, codewords)
    d, M1, M2 = 96, 32, 31
    xt = dg.gaussian_mixture(40000, d, 64, stream=dg.STREAM_TRAIN)
    xb = dg.gaussian_mixture(2500, d, 64, stream=dg.STREAM_BASE)
    out = []
    for nt in (1, 3, 0):
        h = lc.lc_create(lc.lc_default_params(d, M1, M2, use_opq=1, opq_iters=2, kmeans_iters=4, batch_max=256,
                                              n_threads=nt))
        try:
            lc.lc_train(h, xt)
            lc.lc_add(h, xb)
            out.append(lc.lc_export(h, d, M1, M2))
        finally:
            lc.lc_free(h)
    for ex in out[1:]:
        for key in ("R", "C1", "C2", "codes1", "codes2", "beta", "B", "adj0", "levels", "upper_adj"):
            assert np.array_equal(np.asarray(ex[key]), np.asarray(out[0][key])), key


def test_add_u8_equals_add_of_the_same_values():
    d = 32
    xt = dg.sift_like(1500, d, 32, stream=dg.STREAM_TRAIN)
    xb = dg.sift_like(800, d, 32, stream=dg.STREAM_BASE)
    assert np.array_equal(xb, np.round(xb)) and xb.min() >= 0 and xb.max() <= 255
    out = []
    for u8 in (False, True):
        h = lc.lc_create(lc.lc_default_params(d, 16, 8, use_opq=0, kmeans_iters=5))
        try:
            lc.lc_train(h, xt)
            if u8:
                lc.lc_add_u8(h, xb.astype(np.uint8))
            else:
                lc.lc_add(h, xb)
            out.append(lc.lc_export(h, d, 16, 8))
        finally:
            lc.lc_free(h)
    for key in out[0]:
        assert np.array_equal(np.asarray(out[0][key]), np.asarray(out[1][key])), key



@pytest.mark.parametrize("bM,bK", [(4, 16), (3, 1)])
def test_product_codebook_build(bM, bK):
    # the library's product regression codebook (Section 4.3) and 0-byte weights per block
    # (Section 4.2): e0 first in every block, every codeword the blockwise argmin under the
    # library's own codebooks, and (0-byte, trained on every vector) the blockwise least
    # squares of the oracle
    d, M1, M2, n = 48, 16, 16, 1500
    xt = dg.gaussian_mixture(3000, d, 32, stream=dg.STREAM_TRAIN)
    xb = dg.gaussian_mixture(n, d, 32, stream=dg.STREAM_BASE)
    h = lc.lc_create(lc.lc_default_params(d, M1, M2, use_opq=0, kmeans_iters=6, beta_M=bM, beta_K=bK,
                                          beta_iters=3, beta_train_n=n))
    try:
        lc.lc_train(h, xt)
        lc.lc_add(h, xb)
        ex = lc.lc_export(h, d, M1, M2, bM, bK)
    finally:
        lc.lc_free(h)
    B, beta = ex["B"].astype(np.float64), ex["beta"].astype(np.int64)
    assert B.shape == (bM, bK, 9) and beta.shape == (n, bM)
    xr = xb.astype(np.float64) @ ex["R"].astype(np.float64).T
    xh = codec.pq_decode(ex["codes1"], ex["C1"].astype(np.float64), M1) + \
        codec.pq_decode(ex["codes2"], ex["C2"].astype(np.float64), M2)
    G = refine.gmatrix(xh, ex["adj0"], np.arange(n))
    if bK == 1:
        assert not beta.any()
        ref = refine.train_product(G, xr, bM, 1)
        np.testing.assert_allclose(B, ref, rtol=1e-4, atol=1e-5)
        return
    assert np.array_equal(B[:, 0], np.tile(refine.e0(), (bM, 1)))
    best = refine.assign_product(G, xr, B)
    assert (best == beta).mean() > 0.98
    y_lib = refine.reconstruct(G, B, beta)
    y_best = refine.reconstruct(G, B, best)
    e_lib = ((xr - y_lib) ** 2).sum(1)
    assert np.all(e_lib <= ((xr - y_best) ** 2).sum(1) * (1 + 1e-5) + 1e-9)
    assert np.all(e_lib <= ((xr - xh) ** 2).sum(1) * (1 + 1e-5) + 1e-9)
