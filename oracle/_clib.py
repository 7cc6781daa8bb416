"""Compiles and loads the oracle's C helper (``lc_oracle.c``) with gcc.

Test infrastructure only: see the package docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_OUT = os.path.join(_OUT_DIR, "liblc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C code into ``oracle/_lib/liblc_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            L.orc_search.restype = ctypes.c_int
            L.orc_search.argtypes = [i64, i32, i32, i32, P, P, P, P, P, P, P, i32, i32, i32, P, i32, P, P,
                                     ctypes.c_int32, i32, i64, P, i32, i32, i32, i32, i32, P, i32, P, P, P, P, P,
                                     P, P, P, P, P]
            L.orc_dists.restype = ctypes.c_int
            L.orc_dists.argtypes = [i64, i32, i32, i32, P, P, P, P, P, P, P, i32, i32, i32, P, i64, P, i32, P,
                                    P, i32, P, P, P]
            L.orc_trace.restype = ctypes.c_int
            L.orc_trace.argtypes = [P, i32]
            L.orc_build_graph.restype = ctypes.c_int
            L.orc_build_graph.argtypes = [i64, i32, P, P, P, i32, i32, i32, i32, i32, P, P, i64, P,
                                          P, P]
            _lib = L
        return _lib


def ptr(a):
    """Address of a C-contiguous numpy array (or NULL for None)."""
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)
