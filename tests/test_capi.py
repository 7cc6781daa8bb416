"""C ABI checks that need no GPU: the library loads and exports every entry point that
include/lc.h declares; argument and state errors are reported as statuses; import, export
and the file format round-trip; the host build (train + add) produces a well-formed index."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1804_09996_gb300 import lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1804_09996_gb300 import build
    build.build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "lc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L = lc.lib()
    names = header_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lc.EXPORTED) == names


def test_param_validation():
    with pytest.raises(lc.LcError) as e:
        lc.lc_create(lc.lc_default_params(96, 24, 16))
    assert e.value.status == lc.LC_ERR_ARG and "M1" in e.value.message
    with pytest.raises(lc.LcError):
        lc.lc_create(lc.lc_default_params(96, 32, 16, deg=16))
    with pytest.raises(lc.LcError):
        lc.lc_create(lc.lc_default_params(300, 32, 16))
    for bm, bk in ((0, 256), (33, 256), (4, 0), (4, 257)):
        with pytest.raises(lc.LcError) as e:
            lc.lc_create(lc.lc_default_params(96, 32, 16, beta_M=bm, beta_K=bk))
        assert e.value.status == lc.LC_ERR_ARG and "beta_" in e.value.message
    p = lc.lc_default_params(96, 32, 16)
    assert (p.beta_M, p.beta_K) == (1, 256)


def test_state_errors_without_gpu():
    h = lc.lc_create(lc.lc_default_params(16, 16, 8, use_opq=0))
    try:
        with pytest.raises(lc.LcError) as e:
            lc.lc_add(h, np.zeros((3, 16), np.float32))
        assert e.value.status == lc.LC_ERR_STATE
        q = np.zeros((1, 16), np.float32)
        ids = np.zeros((1, 1), np.int32)
        ds = np.zeros((1, 1), np.float32)
        with pytest.raises(lc.LcError) as e:
            lc.lc_search(h, q, 1, lc.lc_default_search_params(1, 8), ids, ds)
        assert e.value.status == lc.LC_ERR_STATE
        with pytest.raises(lc.LcError) as e:
            lc.lc_search(h, q, 1, lc.lc_default_search_params(0, 8), ids, ds)
        assert e.value.status == lc.LC_ERR_ARG
        with pytest.raises(lc.LcError) as e:
            lc.lc_search(h, q, 1, lc.lc_default_search_params(4, 2000), ids, ds)
        assert e.value.status == lc.LC_ERR_ARG
        with pytest.raises(lc.LcError) as e:
            lc.lc_search(h, q, 1, lc.lc_default_search_params(1, 8, order=3), ids, ds)
        assert e.value.status == lc.LC_ERR_ARG and "order" in e.value.message
        for beam in (1, 9):
            with pytest.raises(lc.LcError) as e:
                lc.lc_search(h, q, 1, lc.lc_default_search_params(1, 8, mode=lc.LC_MODE_BATCHED, beam=beam), ids, ds)
            assert e.value.status == lc.LC_ERR_ARG and "beam" in e.value.message
        for bad in (7, 17, -1):
            with pytest.raises(lc.LcError) as e:
                lc.lc_search(h, q, 1, lc.lc_default_search_params(1, 8, spill_log=bad), ids, ds)
            assert e.value.status == lc.LC_ERR_ARG and "spill_log" in e.value.message
        with pytest.raises(lc.LcError) as e:
            lc.lc_train(h, np.zeros((10, 16), np.float32))
        assert e.value.status == lc.LC_ERR_ARG
    finally:
        lc.lc_free(h)


def _import(ix):
    h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2))
    lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0,
                 ix.levels, ix.upper_adj, ix.ep)
    return h


def test_import_export_and_file_roundtrip(mix3k, tmp_path):
    ix, _, _ = mix3k
    h = _import(ix)
    try:
        ex = lc.lc_export(h, ix.d, ix.M1, ix.M2)
        for k in ("R", "C1", "C2", "codes1", "codes2", "beta", "B", "adj0", "levels", "upper_adj"):
            assert np.array_equal(ex[k], getattr(ix, k)), k
        assert ex["ep"] == ix.ep
        path = str(tmp_path / "ix.lc")
        lc.lc_save(h, path)
        h2 = lc.lc_load(path)
        try:
            ex2 = lc.lc_export(h2, ix.d, ix.M1, ix.M2)
            for k in ex:
                assert np.array_equal(np.asarray(ex[k]), np.asarray(ex2[k])), k
        finally:
            lc.lc_free(h2)
    finally:
        lc.lc_free(h)
    bad = tmp_path / "bad.lc"
    bad.write_bytes(b"not an index")
    with pytest.raises(lc.LcError) as e:
        lc.lc_load(str(bad))
    assert e.value.status == lc.LC_ERR_IO
    # a truncated file, trailing bytes, and an upper-row count that disagrees with the levels
    good = (tmp_path / "ix.lc").read_bytes()
    rows_at = 8 + ctypes.sizeof(lc.lc_params) + 8
    rows = int(np.frombuffer(good[rows_at:rows_at + 8], np.int64)[0])
    assert rows == len(ix.upper_adj) > 0
    fewer = good[:rows_at] + np.int64(rows - 1).tobytes() + good[rows_at + 8:-ix.upper_adj.shape[1] * 4]
    for blob, words in ((good[:-7], "truncated"), (good + b"\0", "after the index"),
                        (fewer, "upper rows")):
        bad.write_bytes(blob)
        with pytest.raises(lc.LcError) as e:
            lc.lc_load(str(bad))
        assert e.value.status == lc.LC_ERR_IO and words in e.value.message, e.value.message


def test_import_rejects_bad_graphs(mix3k):
    ix, _, _ = mix3k
    h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2))
    try:
        adj = ix.adj0.copy()
        adj[5, 0] = ix.N + 3
        with pytest.raises(lc.LcError) as e:
            lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, adj,
                         ix.levels, ix.upper_adj, ix.ep)
        assert e.value.status == lc.LC_ERR_ARG
        ep_bad = int(np.flatnonzero(ix.levels == 0)[0])
        with pytest.raises(lc.LcError):
            lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ix.beta, ix.B, ix.adj0,
                         ix.levels, ix.upper_adj, ep_bad)
    finally:
        lc.lc_free(h)


def test_search_ex_argument_errors_without_gpu(mix3k):
    # both checks happen on the host before any device work
    ix, _, xq = mix3k
    h = _import(ix)
    try:
        q = np.ascontiguousarray(xq[:4], np.float32)
        ids = np.empty((4, 10), np.int32)
        ds = np.empty((4, 10), np.float32)
        sp = lc.lc_default_search_params(10, 64)
        with pytest.raises(lc.LcError) as e:
            lc.lc_search_ex(h, q, 7, 4, sp, None, ids, ds)
        assert e.value.status == lc.LC_ERR_ARG and "query type" in e.value.message
        for bad in (0, 65):
            efq = np.array([16, bad, 32, 64], np.int32)
            with pytest.raises(lc.LcError) as e:
                lc.lc_search_ex(h, q, lc.LC_QUERY_F32, 4, sp, efq, ids, ds)
            assert e.value.status == lc.LC_ERR_ARG and "query 1" in e.value.message
        # codebook precisions: FP32, FP16 and the table form; anything else is refused
        for bad in (-1, lc.LC_LUT_TABLE + 1):
            with pytest.raises(lc.LcError) as e:
                lc.lc_search(h, q, 4, lc.lc_default_search_params(10, 64, lut_prec=bad), ids, ds)
            assert e.value.status == lc.LC_ERR_ARG and "lut_prec" in e.value.message
    finally:
        lc.lc_free(h)


@pytest.mark.parametrize("bM,bK", [(4, 16), (3, 1)])
def test_product_codebook_import_export_and_file(mix3k, tmp_path, bM, bK):
    # product regression codebook (beta [n][bM], B [bM][bK][9]) and the 0-byte weights
    from oracle.index import with_regression
    ix, _, _ = mix3k
    ixp = with_regression(ix, bM, bK, beta_train_n=1000, beta_iters=2)
    h = lc.lc_create(lc.lc_default_params(ix.d, ix.M1, ix.M2, beta_M=bM, beta_K=bK))
    try:
        lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, ixp.beta, ixp.B, ix.adj0,
                     ix.levels, ix.upper_adj, ix.ep)
        ex = lc.lc_export(h, ix.d, ix.M1, ix.M2, bM, bK)
        assert np.array_equal(ex["beta"], ixp.beta) and np.array_equal(ex["B"], ixp.B)
        path = str(tmp_path / "p.lc")
        lc.lc_save(h, path)
        h2 = lc.lc_load(path)
        try:
            ex2 = lc.lc_export(h2, ix.d, ix.M1, ix.M2, bM, bK)
            for k in ex:
                assert np.array_equal(np.asarray(ex[k]), np.asarray(ex2[k])), k
        finally:
            lc.lc_free(h2)
        if bK > 1:
            bad = ixp.beta.copy()
            bad[5, 1] = bK
            with pytest.raises(lc.LcError) as e:
                lc.lc_import(h, ix.N, ix.R, ix.C1, ix.C2, ix.codes1, ix.codes2, bad, ixp.B, ix.adj0,
                             ix.levels, ix.upper_adj, ix.ep)
            assert e.value.status == lc.LC_ERR_ARG and "codeword" in e.value.message
    finally:
        lc.lc_free(h)


def test_plan_argument_errors_without_gpu(mix3k):
    ix, _, _ = mix3k
    h = _import(ix)
    try:
        sp = lc.lc_default_search_params(10, 64)
        for nq_max, qt in ((0, lc.LC_QUERY_F32), (16, 5)):
            with pytest.raises(lc.LcError) as e:
                lc.lc_plan_create(h, nq_max, sp, qt)
            assert e.value.status == lc.LC_ERR_ARG
        bad = lc.lc_default_search_params(10, 64, warps=17)
        with pytest.raises(lc.LcError) as e:
            lc.lc_plan_create(h, 16, bad)
        assert e.value.status == lc.LC_ERR_ARG and "warps" in e.value.message
    finally:
        lc.lc_free(h)


def test_autotune_argument_errors_without_gpu(mix3k):
    ix, _, xq = mix3k
    h = _import(ix)
    try:
        for kw in (dict(k=0), dict(max_beam=9), dict(reps=0), dict(ef=2000)):
            with pytest.raises(lc.LcError) as e:
                lc.lc_autotune(h, xq[:10], **kw)
            assert e.value.status == lc.LC_ERR_ARG
    finally:
        lc.lc_free(h)


def test_gpu_build_without_gpu_leaves_index_untouched():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = lc.lc_create(lc.lc_default_params(16, 16, 8, use_opq=0, kmeans_iters=2, build_gpu=1))
    try:
        rng = np.random.default_rng(0)
        lc.lc_train(h, rng.standard_normal((400, 16)).astype(np.float32))
        with pytest.raises(lc.LcError) as e:
            lc.lc_add(h, rng.standard_normal((50, 16)).astype(np.float32))
        assert e.value.status == lc.LC_ERR_CUDA and "CUDA device" in e.value.message
        assert lc.lc_size(h) == 0
    finally:
        lc.lc_free(h)
