"""Seeded synthetic inputs shaped like the workloads of Link and Code (Douze,
Sablayrolles, Jegou, CVPR 2018).

The paper evaluates on Deep1B (unit-norm 96-d CNN descriptors) and BIGANN (SIFT
vectors), Section 5.  Neither dataset is available here, so these generators stand
in for them.  This module holds no arithmetic of the method itself: it only draws
random vectors.  Both the CUDA path and the CPU oracle are fed from it.

Every draw is counter-based: rows are produced in chunks of ``CHUNK`` rows, and
chunk ``c`` of stream ``s`` under seed ``seed`` comes from a Philox generator keyed
by ``(seed, s, c)``.  Any row range can therefore be regenerated on its own, and a
database of 50M rows can be streamed chunk by chunk.

Streams used by convention: 0 = mixture centres / profiles, 1 = training set,
2 = database, 3 = queries, 4 = per-query search parameters.
"""
from __future__ import annotations

import numpy as np

CHUNK = 1 << 16
SEED = 1804
STREAM_CENTRES, STREAM_TRAIN, STREAM_BASE, STREAM_QUERY, STREAM_PARAMS = 0, 1, 2, 3, 4


def _rng(seed: int, stream: int, chunk: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, stream, chunk])))


def _chunked(n: int, start: int, seed: int, stream: int, draw):
    """Assemble rows [start, start+n) from per-chunk draws ``draw(rng, rows)``."""
    out = []
    i = start
    end = start + n
    while i < end:
        c = i // CHUNK
        lo = c * CHUNK
        block = draw(_rng(seed, stream, c), CHUNK)
        a = i - lo
        b = min(end - lo, CHUNK)
        out.append(block[a:b])
        i = lo + b
    if not out:
        return None
    return np.concatenate(out, axis=0)


def mixture_centres(d: int, n_centres: int, seed: int = SEED) -> np.ndarray:
    """Centres mu_m ~ N(0, I/d), float64 [n_centres][d]."""
    g = _rng(seed, STREAM_CENTRES, 0)
    return g.standard_normal((n_centres, d)) / np.sqrt(d)


def gaussian_mixture(n: int, d: int = 96, n_centres: int = 64, sigma: float = 0.6,
                     seed: int = SEED, stream: int = STREAM_BASE, start: int = 0) -> np.ndarray:
    """Deep1B stand-in: x = mu_m + sigma * N(0, I/d), m uniform, then L2-normalised.

    Returns float32 [n][d].  Rows are a pure function of (seed, stream, row index).
    """
    mu = mixture_centres(d, n_centres, seed)

    def draw(g, rows):
        m = g.integers(0, n_centres, size=rows)
        z = g.standard_normal((rows, d)) / np.sqrt(d)
        x = mu[m] + sigma * z
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        return x.astype(np.float32)

    out = _chunked(n, start, seed, stream, draw)
    return np.zeros((0, d), np.float32) if out is None else out


def sphere(n: int, d: int = 96, seed: int = SEED, stream: int = STREAM_BASE, start: int = 0) -> np.ndarray:
    """Directions drawn uniformly on the unit sphere (normalised N(0, I)), float32 [n][d]:
    the mixture without any cluster structure, a stress input on which graph walks are long
    (every query sees a flat distance landscape)."""
    def draw(g, rows):
        x = g.standard_normal((rows, d))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        return x.astype(np.float32)

    out = _chunked(n, start, seed, stream, draw)
    return np.zeros((0, d), np.float32) if out is None else out


def sift_profiles(d: int = 128, n_profiles: int = 1024, seed: int = SEED) -> np.ndarray:
    g = _rng(seed, STREAM_CENTRES, 1)
    return g.gamma(0.5, 40.0, size=(n_profiles, d))


def sift_like(n: int, d: int = 128, n_profiles: int = 1024, seed: int = SEED,
              stream: int = STREAM_BASE, start: int = 0) -> np.ndarray:
    """BIGANN stand-in: non-negative, heavy-tailed, integer-valued, many zeros.

    x_t = min(255, floor(mu_{m,t} * E_t)), mu ~ Gamma(0.5, 40), E ~ Exp(1).
    Returns uint8 [n][d].
    """
    mu = sift_profiles(d, n_profiles, seed)

    def draw(g, rows):
        m = g.integers(0, n_profiles, size=rows)
        e = g.standard_exponential((rows, d))
        return np.minimum(255.0, np.floor(mu[m] * e)).astype(np.uint8)

    out = _chunked(n, start, seed, stream, draw)
    return np.zeros((0, d), np.uint8) if out is None else out


def uneven_ef(n: int, choices=(16, 32, 64, 128, 256), seed: int = SEED, start: int = 0) -> np.ndarray:
    """Per-query efSearch drawn uniformly from ``choices`` (int32 [n])."""
    ch = np.asarray(choices, np.int32)

    def draw(g, rows):
        return ch[g.integers(0, len(ch), size=rows)]

    out = _chunked(n, start, seed, STREAM_PARAMS, draw)
    return np.zeros((0,), np.int32) if out is None else out


# Named workloads: (database size, queries, dim, M1, M2, generator kwargs).
WORKLOADS = {
    # 10k database / 1k queries, 96-d mixture of 64 Gaussians; PQ16 + residual PQ16.
    "mix10k": dict(n_base=10_000, n_query=1_000, n_train=10_000, d=96, M1=16, M2=16,
                   use_opq=False, kind="mixture", n_centres=64),
    # 1M database / 10k queries per launch, 1,024 centres; OPQ32 + residual PQ31 = 64 B/vector.
    "mix1m": dict(n_base=1_000_000, n_query=10_000, n_train=100_000, d=96, M1=32, M2=31,
                  use_opq=True, kind="mixture", n_centres=1024),
    # 10M SIFT-like uint8, 128-d; PQ64 + residual PQ63 = 128 B/vector.
    "sift10m": dict(n_base=10_000_000, n_query=100_000, n_train=200_000, d=128, M1=64, M2=63,
                    use_opq=True, kind="sift", n_centres=1024),
}


def make(kind: str, n: int, d: int, n_centres: int, stream: int, seed: int = SEED,
         start: int = 0) -> np.ndarray:
    """Rows of a named generator as float32 (SIFT-like values are converted exactly)."""
    if kind == "mixture":
        return gaussian_mixture(n, d, n_centres, seed=seed, stream=stream, start=start)
    if kind == "sift":
        return sift_like(n, d, n_centres, seed=seed, stream=stream, start=start).astype(np.float32)
    raise ValueError(f"unknown generator kind {kind!r}")
