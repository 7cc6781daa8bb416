"""Thin ctypes binding of liblc.so: the entry points of include/lc.h under the same names,
with argument marshalling only (numpy arrays for host memory, torch tensors for device
memory).  Every step of the search runs in the library's CUDA kernels; if the library is
not built this module raises instead of doing the work any other way.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblc.so")

LC_OK, LC_ERR_ARG, LC_ERR_OOM, LC_ERR_STATE, LC_ERR_CUDA = 0, 1, 2, 3, 4
LC_ERR_TIMEOUT, LC_ERR_BUDGET, LC_ERR_IO, LC_ERR_CAPACITY = 5, 6, 7, 8
LC_MODE_PLAIN, LC_MODE_BATCHED = 0, 1
LC_LUT_FP32, LC_LUT_FP16, LC_LUT_TABLE = 0, 1, 2
LC_QUERY_F32, LC_QUERY_U8 = 0, 1
LC_ORDER_AUTO, LC_ORDER_NEVER, LC_ORDER_ALWAYS = 0, 1, 2

EXPORTED = [
    "lc_default_params", "lc_default_search_params", "lc_create", "lc_train", "lc_add", "lc_add_u8",
    "lc_search", "lc_search_ex",
    "lc_import", "lc_size", "lc_upper_rows", "lc_export", "lc_save", "lc_load", "lc_profile",
    "lc_profile_read", "lc_profile_phases", "lc_free", "lc_last_error", "lc_search_walk_noalloc",
    "lc_serve_open", "lc_serve_submit", "lc_serve_poll", "lc_serve_close", "lc_merge_topk",
    "lc_plan_create", "lc_plan_buffers", "lc_plan_run", "lc_plan_free", "lc_autotune",
]

# void (*lc_request_cb)(void *user, uint64_t req_id, lc_status status, const int32_t *ids,
#                       const float *dists, int32_t nq, int32_t k)
LC_REQUEST_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                 ctypes.c_int32, ctypes.c_int32)


class LcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lc status {status}: {message}")
        self.status = status
        self.message = message


class lc_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "d", "M1", "M2", "use_opq", "deg", "deg_upper", "level_ratio", "ef_construction",
        "beta_train_n", "beta_iters", "kmeans_iters", "opq_iters", "batch_max", "n_threads")] + [
        ("seed", ctypes.c_uint64), ("beta_M", ctypes.c_int), ("beta_K", ctypes.c_int), ("build_gpu", ctypes.c_int)]


class lc_search_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("k", "ef", "shortlist", "lut_prec", "mode", "visited_log", "beam", "max_dist", "warps",
                                                     "walk_full", "order", "spill_log")]


class lc_tune_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("k", "ef", "allow_fp16", "max_beam", "reps", "batch")]


class lc_tune_result(ctypes.Structure):
    _fields_ = [("sp", lc_search_params)] + [(n, ctypes.c_float) for n in ("ms", "recall", "target", "base_ms")] + [
        ("tried", ctypes.c_int)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if it has not been built (``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                           "(the search has no other implementation)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "lc_default_params": (None, [P, I, I, I]),
        "lc_default_search_params": (None, [P, I, I]),
        "lc_create": (I, [P, P]),
        "lc_train": (I, [P, P, I64]),
        "lc_add": (I, [P, P, I64]),
        "lc_add_u8": (I, [P, P, I64]),
        "lc_search": (I, [P, P, I64, P, P, P, P, P]),
        "lc_search_ex": (I, [P, P, I, I64, P, P, P, P, P, P]),
        "lc_import": (I, [P, I64, P, P, P, P, P, P, P, P, P, P, ctypes.c_int32]),
        "lc_size": (I64, [P]),
        "lc_upper_rows": (I64, [P]),
        "lc_export": (I, [P, P, P, P, P, P, P, P, P, P, P, P]),
        "lc_save": (I, [P, ctypes.c_char_p]),
        "lc_load": (I, [ctypes.c_char_p, P]),
        "lc_profile": (I, [P, I]),
        "lc_search_walk_noalloc": (I, [P, P, I64, I, I, P, P, P, P]),
        "lc_serve_open": (I, [P, ctypes.c_size_t, I, I, P]),
        "lc_merge_topk": (I, [P, P, I, I64, I, P, P, P, P]),
        "lc_serve_submit": (I, [P, P, ctypes.c_int32, P, LC_REQUEST_CB, P, P]),
        "lc_serve_poll": (I, [P, I, P]),
        "lc_serve_close": (I, [P]),
        "lc_profile_read": (I, [P, P, P]),
        "lc_profile_phases": (I, [P, P, P, P, P]),
        "lc_autotune": (I, [P, P, I64, P, P, P]),
        "lc_plan_create": (I, [P, I64, P, I, I, P]),
        "lc_plan_buffers": (I, [P, P, P, P, P, P]),
        "lc_plan_run": (I, [P, I64, P]),
        "lc_plan_free": (None, [P]),
        "lc_free": (None, [P]),
        "lc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def lc_last_error() -> str:
    return lib().lc_last_error().decode()


def _check(status: int):
    if status != LC_OK:
        raise LcError(status, lc_last_error())


def _ptr(a):
    """Address of a C-contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported buffer type {type(a)!r}")


def lc_default_params(d: int, M1: int, M2: int, **overrides) -> lc_params:
    p = lc_params()
    lib().lc_default_params(ctypes.byref(p), d, M1, M2)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def lc_default_search_params(k: int, ef: int, **overrides) -> lc_search_params:
    p = lc_search_params()
    lib().lc_default_search_params(ctypes.byref(p), k, ef)
    for key, v in overrides.items():
        setattr(p, key, v)
    return p


def lc_create(params: lc_params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().lc_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def lc_train(ix, xt: np.ndarray):
    xt = np.ascontiguousarray(xt, np.float32)
    _check(lib().lc_train(ix, _ptr(xt), xt.shape[0]))


def lc_add(ix, x: np.ndarray):
    x = np.ascontiguousarray(x, np.float32)
    _check(lib().lc_add(ix, _ptr(x), x.shape[0]))


def lc_add_u8(ix, x: np.ndarray):
    x = np.ascontiguousarray(x, np.uint8)
    _check(lib().lc_add_u8(ix, _ptr(x), x.shape[0]))


def lc_search(ix, q, nq: int, sp: lc_search_params, ids, dists, stats=None, stream=None):
    """q [nq][d] float32, ids [nq][k] int32, dists [nq][k] float32, stats [nq][3] int32 or
    None: all numpy (host) or all torch CUDA tensors (device; queued on ``stream``, a
    torch.cuda.Stream, an integer handle, or None for the current default stream)."""
    s = stream
    if s is not None and hasattr(s, "cuda_stream"):
        s = s.cuda_stream
    _check(lib().lc_search(ix, _ptr(q), nq, ctypes.byref(sp), _ptr(ids), _ptr(dists), _ptr(stats),
                           ctypes.c_void_p(s) if s else None))


def lc_search_ex(ix, q, qtype: int, nq: int, sp: lc_search_params, ef, ids, dists, stats=None, stream=None):
    """lc_search with uint8 queries (qtype LC_QUERY_U8, q [nq][d] uint8) and/or per-query
    efSearch (ef [nq] int32, or None); buffers as lc_search."""
    s = stream
    if s is not None and hasattr(s, "cuda_stream"):
        s = s.cuda_stream
    _check(lib().lc_search_ex(ix, _ptr(q), qtype, nq, ctypes.byref(sp), _ptr(ef), _ptr(ids), _ptr(dists),
                              _ptr(stats), ctypes.c_void_p(s) if s else None))


def lc_search_walk_noalloc(ix, q, nq: int, k: int, ef: int, ids, dists, stats=None, stream=None):
    """The walk of lc_search without refinement, with no device allocation (device tensors
    only; see include/lc.h for the requirements)."""
    s = stream
    if s is not None and hasattr(s, "cuda_stream"):
        s = s.cuda_stream
    _check(lib().lc_search_walk_noalloc(ix, _ptr(q), nq, k, ef, _ptr(ids), _ptr(dists), _ptr(stats),
                                        ctypes.c_void_p(s) if s else None))


def lc_merge_topk(ids, dists, S: int, nq: int, k: int, id_offsets, ids_out, dists_out, stream=None):
    """ids/dists: device tensors [S][nq][k]; id_offsets: sequence of S ints; outputs [nq][k]."""
    off = np.ascontiguousarray(np.asarray(id_offsets, np.int64))
    s = stream
    if s is not None and hasattr(s, "cuda_stream"):
        s = s.cuda_stream
    _check(lib().lc_merge_topk(_ptr(ids), _ptr(dists), S, nq, k, _ptr(off), _ptr(ids_out), _ptr(dists_out),
                               ctypes.c_void_p(s) if s else None))


def make_request_cb(fn):
    """Wraps fn(req_id, status, ids, dists) into an lc_request_cb; ids/dists are copied into
    numpy arrays ([nq][k]) when status is LC_OK, else None.  Keep the returned object alive
    until the request has completed."""
    def _cb(user, req_id, status, ids, dists, nq, k):
        if status == LC_OK:
            i = np.ctypeslib.as_array(ids, shape=(nq, k)).copy()
            d = np.ctypeslib.as_array(dists, shape=(nq, k)).copy()
        else:
            i = d = None
        fn(int(req_id), int(status), i, d)
    return LC_REQUEST_CB(_cb)


def lc_serve_open(ix, device_budget_bytes: int, max_inflight: int, max_request: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().lc_serve_open(ix, device_budget_bytes, max_inflight, max_request, ctypes.byref(h)))
    return h


def lc_serve_submit(srv, q: np.ndarray, sp: lc_search_params, cb) -> int:
    q = np.ascontiguousarray(q, np.float32)
    rid = ctypes.c_uint64()
    _check(lib().lc_serve_submit(srv, _ptr(q), q.shape[0], ctypes.byref(sp), cb, None, ctypes.byref(rid)))
    return int(rid.value)


def lc_serve_poll(srv, timeout_ms: int = 0) -> int:
    n = ctypes.c_int()
    _check(lib().lc_serve_poll(srv, timeout_ms, ctypes.byref(n)))
    return int(n.value)


def lc_serve_close(srv):
    _check(lib().lc_serve_close(srv))


def lc_import(ix, n, R, C1, C2, codes1, codes2, beta, B, adj0, levels, upper_adj, ep: int):
    arrs = [np.ascontiguousarray(R, np.float32), np.ascontiguousarray(C1, np.float32),
            np.ascontiguousarray(C2, np.float32), np.ascontiguousarray(codes1, np.uint8),
            np.ascontiguousarray(codes2, np.uint8), np.ascontiguousarray(beta, np.uint8),
            np.ascontiguousarray(B, np.float32), np.ascontiguousarray(adj0, np.int32),
            np.ascontiguousarray(levels, np.int32), np.ascontiguousarray(upper_adj, np.int32)]
    ptrs = [_ptr(a) if a.size else None for a in arrs]
    for i in range(3):          # rotation and codebooks are never empty
        ptrs[i] = _ptr(arrs[i])
    ptrs[6] = _ptr(arrs[6])
    _check(lib().lc_import(ix, n, *ptrs, ep))


def lc_size(ix) -> int:
    return int(lib().lc_size(ix))


def lc_upper_rows(ix) -> int:
    return int(lib().lc_upper_rows(ix))


def lc_export(ix, d: int, M1: int, M2: int, beta_M: int = 1, beta_K: int = 256) -> dict:
    """The index arrays (layouts of lc_import).  With one regression block beta is [n] and B
    [beta_K][9]; with beta_M blocks, [n][beta_M] and [beta_M][beta_K][9]."""
    n, rows = lc_size(ix), lc_upper_rows(ix)
    out = dict(R=np.empty((d, d), np.float32), C1=np.empty((256, d), np.float32),
               C2=np.empty((256, d), np.float32), codes1=np.empty((n, M1), np.uint8),
               codes2=np.empty((n, M2), np.uint8),
               beta=np.empty(n, np.uint8) if beta_M == 1 else np.empty((n, beta_M), np.uint8),
               B=np.empty((beta_K, 9) if beta_M == 1 else (beta_M, beta_K, 9), np.float32),
               adj0=np.empty((n, 32), np.int32),
               levels=np.empty(n, np.int32), upper_adj=np.empty((rows, 32), np.int32))
    ep = ctypes.c_int32()
    order = ["R", "C1", "C2", "codes1", "codes2", "beta", "B", "adj0", "levels", "upper_adj"]
    _check(lib().lc_export(ix, *[_ptr(out[k]) if out[k].size else None for k in order], ctypes.byref(ep)))
    out["ep"] = int(ep.value)
    return out


def lc_save(ix, path: str):
    _check(lib().lc_save(ix, path.encode()))


def lc_load(path: str) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().lc_load(path.encode(), ctypes.byref(h)))
    return h


def lc_profile(ix, enable: bool):
    _check(lib().lc_profile(ix, 1 if enable else 0))


def lc_profile_read(ix):
    """(walk_ms, refine_ms) of the last profiled search."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(lib().lc_profile_read(ix, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lc_profile_phases(ix):
    """(rotate_ms, descent_ms, level0_ms, refine_ms) of the last profiled search."""
    v = [ctypes.c_float() for _ in range(4)]
    _check(lib().lc_profile_phases(ix, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lc_free(ix):
    if ix:
        lib().lc_free(ix)


class _DeviceView:
    """A device buffer described by __cuda_array_interface__ (for torch.as_tensor)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def lc_plan_create(ix, nq_max: int, sp: lc_search_params, qtype: int = LC_QUERY_F32,
                   per_query_ef: bool = False) -> ctypes.c_void_p:
    pl = ctypes.c_void_p()
    _check(lib().lc_plan_create(ix, nq_max, ctypes.byref(sp), qtype, int(per_query_ef), ctypes.byref(pl)))
    return pl


def lc_plan_buffers(pl) -> dict:
    """Device addresses of the plan's buffers (ef is 0 without per-query efSearch)."""
    ptrs = [ctypes.c_void_p() for _ in range(5)]
    _check(lib().lc_plan_buffers(pl, *[ctypes.byref(p) for p in ptrs]))
    return {n: int(p.value or 0) for n, p in zip(("q", "ef", "ids", "dists", "stats"), ptrs)}


def lc_plan_tensors(pl, nq_max: int, d: int, k: int, qtype: int = LC_QUERY_F32) -> dict:
    """The plan's buffers as torch CUDA tensors (views, no copy): q, ef (or None), ids,
    dists, stats, each with nq_max rows."""
    import torch
    b = lc_plan_buffers(pl)
    view = lambda ptr, shape, ts: torch.as_tensor(_DeviceView(ptr, shape, ts), device="cuda")  # noqa: E731
    return {"q": view(b["q"], (nq_max, d), "|u1" if qtype == LC_QUERY_U8 else "<f4"),
            "ef": view(b["ef"], (nq_max,), "<i4") if b["ef"] else None,
            "ids": view(b["ids"], (nq_max, k), "<i4"), "dists": view(b["dists"], (nq_max, k), "<f4"),
            "stats": view(b["stats"], (nq_max, 3), "<i4")}


def lc_plan_run(pl, nq: int, stream=None):
    s = stream
    if s is not None and hasattr(s, "cuda_stream"):
        s = s.cuda_stream
    _check(lib().lc_plan_run(pl, nq, ctypes.c_void_p(s) if s else None))


def lc_plan_free(pl):
    lib().lc_plan_free(pl)


def lc_autotune(ix, q: np.ndarray, gt=None, k: int = 10, ef: int = 64, allow_fp16: bool = True,
                max_beam: int = 8, reps: int = 3, batch: int = 0) -> lc_tune_result:
    """Tune the search on a host sample q [n][d] (float32) with optional exact neighbour ids
    gt [n], timing batches of ``batch`` queries; returns the lc_tune_result (include/lc.h)."""
    q = np.ascontiguousarray(q, np.float32)
    g = None if gt is None else np.ascontiguousarray(gt, np.int32)
    tp = lc_tune_params(k=k, ef=ef, allow_fp16=int(allow_fp16), max_beam=max_beam, reps=reps, batch=batch)
    out = lc_tune_result()
    _check(lib().lc_autotune(ix, _ptr(q), q.shape[0], _ptr(g), ctypes.byref(tp), ctypes.byref(out)))
    return out
