"""HNSW graph of the oracle: level draws and the insertion build (through the C helper).

Test infrastructure only (see the package docstring).

Paper passages: nested layers with geometric sizes, one point in the top layer, the
whole set in the base layer, a neighbour graph per layer (Section 2); degree 32 and a
size ratio of 30 between consecutive layers (Section 4.1); vectors added by batches, the
inserted vector compared exactly against the decoded indexed vectors (Sections 4.1, 5.1).

Level of node i: floor(-ln(U_i) / ln 30), U_i in (0, 1] drawn by SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) as the i-th
output of the generator seeded with ``seed``: z = (seed + (i+1) * 0x9E3779B97F4A7C15) mod
2^64 mixed by the published finaliser, U = ((z >> 11) + 1) / 2^53.  Levels are capped at 15.
"""
from __future__ import annotations

import math

import numpy as np

from ._clib import lib, ptr

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MAX_LEVEL = 15


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """i-th outputs of SplitMix64 seeded with ``seed`` (uint64 arithmetic mod 2^64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(idx, np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def levels(n: int, seed: int, ratio: float = 30.0, start: int = 0) -> np.ndarray:
    z = splitmix64(seed, np.arange(start, start + n, dtype=np.uint64))
    u = ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    lev = np.floor(-np.log(u) / math.log(ratio)).astype(np.int32)
    return np.minimum(lev, MAX_LEVEL).astype(np.int32)


def upper_offsets(lev: np.ndarray):
    """Row offset of each node's level-1 row in the upper adjacency (-1 for level 0).
    Node i with level L_i >= 1 owns rows off_i .. off_i + L_i - 1 (level l at off_i + l - 1)."""
    lev = np.asarray(lev, np.int64)
    off = np.full(lev.shape[0], -1, np.int32)
    has = lev > 0
    csum = np.concatenate([[0], np.cumsum(lev)[:-1]])
    off[has] = csum[has].astype(np.int32)
    return off, int(lev.sum())


def build_graph(xr: np.ndarray, xh: np.ndarray, lev: np.ndarray, deg: int = 32,
                deg_up: int = 32, efc: int = 40, batch_max: int = 1, batch_div: int = 16):
    """Insert all points; returns (adj0 [N][deg], upper_off [N], upper_adj [rows][deg_up],
    ep, max_level).  batch_max = 1 gives sequential insertion."""
    xr = np.ascontiguousarray(xr, np.float64)
    xh = np.ascontiguousarray(xh, np.float64)
    lev = np.ascontiguousarray(lev, np.int32)
    N, d = xr.shape
    off, rows = upper_offsets(lev)
    adj0 = np.empty((N, deg), np.int32)
    upper_adj = np.empty((max(rows, 0), deg_up), np.int32)
    ep = np.zeros(1, np.int32)
    ml = np.zeros(1, np.int32)
    rc = lib().orc_build_graph(N, d, ptr(xr), ptr(xh), ptr(lev), deg, deg_up, efc, batch_max,
                               batch_div, ptr(adj0), ptr(off), rows,
                               ptr(upper_adj) if rows > 0 else None, ptr(ep), ptr(ml))
    if rc != 0:
        raise RuntimeError(f"orc_build_graph failed ({rc})")
    return adj0, off, upper_adj, int(ep[0]), int(ml[0])
