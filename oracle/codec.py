"""Codec of the oracle: k-means, product quantisation, OPQ rotation and the two-level
residual codec, in float64.

Test infrastructure only (see the package docstring).

Paper passages followed:
  * product quantiser "PQ M x 8": M sub-vectors, 256 centroids each, 1 byte per
    sub-vector (Section 3.3, notation of Table 1);
  * OPQ: an orthogonal rotation learned to reduce the PQ error, applied before encoding
    (Section 3.3, and Section 5.1 "systematically perform a rotation");
  * two-level residual codec: the second level encodes x - c1(x) (Section 3.3, and
    Section 4.1 "two-level encodings"), so the reconstruction is q(x) = c1(x) + c2(x - c1(x)).

The paper is silent on the k-means details; the readings used here are: initial centres
are a seeded sample of the points without replacement; a fixed number of Lloyd
iterations; ties go to the lowest centroid index; an empty cluster is re-seeded with the
point of the largest cluster that is furthest from its centre.  M need not divide d: the
first (d mod M) sub-spaces get ceil(d/M) dimensions and the rest floor(d/M).
"""
from __future__ import annotations

import numpy as np

KSUB = 256


def splits(d: int, M: int):
    """(offsets, lengths) of the M contiguous sub-spaces of R^d."""
    base, extra = divmod(d, M)
    lens = [base + (1 if j < extra else 0) for j in range(M)]
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(int).tolist()
    return offs, lens


def sqdist(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Squared L2 distances [n][K] in float64, ||x||^2 - 2 x.c + ||c||^2 (clamped at 0).
    Used for training and encoding only, where the argmin is all that matters."""
    X = np.asarray(X, np.float64)
    C = np.asarray(C, np.float64)
    D = (X * X).sum(1)[:, None] - 2.0 * (X @ C.T) + (C * C).sum(1)[None, :]
    return np.maximum(D, 0.0)


def assign(X: np.ndarray, C: np.ndarray):
    """Nearest centre per row: (index, squared distance); ties go to the lowest index.
    The row constant ||x||^2 does not change the argmin and is added back afterwards."""
    X = np.asarray(X, np.float64)
    C = np.asarray(C, np.float64)
    D = (C * C).sum(1)[None, :] - 2.0 * (X @ C.T)
    a = np.argmin(D, axis=1)
    dmin = D[np.arange(X.shape[0]), a] + (X * X).sum(1)
    return a, np.maximum(dmin, 0.0)


def kmeans(X: np.ndarray, K: int, niter: int = 25, seed: int = 0, init: np.ndarray | None = None):
    """Lloyd's k-means in float64.  Returns centres [K][dim]."""
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    if init is not None:
        C = np.array(init, np.float64, copy=True)
    else:
        g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 77])))
        if n >= K:
            C = X[np.sort(g.choice(n, K, replace=False))].copy()
        else:
            C = X[g.integers(0, n, size=K)].copy()
    for _ in range(niter):
        a, dmin = assign(X, C)
        counts = np.bincount(a, minlength=K)
        sums = np.stack([np.bincount(a, weights=X[:, t], minlength=K) for t in range(X.shape[1])], 1)
        nz = counts > 0
        C[nz] = sums[nz] / counts[nz, None]
        for e in np.flatnonzero(~nz):
            big = int(np.argmax(counts))
            members = np.flatnonzero(a == big)
            if members.size < 2:
                continue
            far = members[np.argmax(dmin[members])]
            C[e] = X[far]
            # the moved point leaves its cluster
            a[far] = e
            counts[big] -= 1
            counts[e] = 1
            dmin[far] = 0.0
    return C


def pq_train(X: np.ndarray, M: int, niter: int = 25, seed: int = 0, init: np.ndarray | None = None):
    """Per-sub-space k-means with 256 centres.  Returns full-width centroids [256][d]:
    row c holds centroid c of every sub-space, each in its own block of coordinates."""
    X = np.asarray(X, np.float64)
    d = X.shape[1]
    offs, lens = splits(d, M)
    C = np.zeros((KSUB, d))
    for j in range(M):
        o, l = offs[j], lens[j]
        C[:, o:o + l] = kmeans(X[:, o:o + l], KSUB, niter, seed + 1000 * j,
                               None if init is None else init[:, o:o + l])
    return C


def pq_encode(X: np.ndarray, C: np.ndarray, M: int) -> np.ndarray:
    """Codes [n][M] uint8: per sub-space the nearest of the 256 centroids."""
    X = np.asarray(X, np.float64)
    offs, lens = splits(X.shape[1], M)
    codes = np.empty((X.shape[0], M), np.uint8)
    for j in range(M):
        o, l = offs[j], lens[j]
        codes[:, j] = assign(X[:, o:o + l], C[:, o:o + l])[0]
    return codes


def pq_decode(codes: np.ndarray, C: np.ndarray, M: int) -> np.ndarray:
    d = C.shape[1]
    offs, lens = splits(d, M)
    out = np.empty((codes.shape[0], d))
    for j in range(M):
        o, l = offs[j], lens[j]
        out[:, o:o + l] = C[codes[:, j].astype(np.int64), o:o + l]
    return out


def opq_train(X: np.ndarray, M: int, n_outer: int = 10, niter_final: int = 25, seed: int = 0):
    """Non-parametric OPQ: alternate a PQ step in the rotated space with the orthogonal
    Procrustes update of the rotation (R = U V^T from the SVD of sum_i xhat_i x_i^T).
    Returns (R [d][d], C [256][d]) with encoding done on R x."""
    X = np.asarray(X, np.float64)
    d = X.shape[1]
    R = np.eye(d)
    C = pq_train(X, M, niter=4, seed=seed)
    for _ in range(n_outer):
        Xr = X @ R.T
        C = pq_train(Xr, M, niter=1, seed=seed, init=C)
        Y = pq_decode(pq_encode(Xr, C, M), C, M)
        U, _, Vt = np.linalg.svd(Y.T @ X)
        R = U @ Vt
    C = pq_train(X @ R.T, M, niter=niter_final, seed=seed, init=C)
    return R, C


def train_codec(xt: np.ndarray, M1: int, M2: int, use_opq: bool, seed: int = 0,
                niter: int = 25, n_outer: int = 10):
    """Two-level codec.  Level 1: (O)PQ M1 x 8 on x' = R x.  Level 2: PQ M2 x 8 on the
    level-1 residual x' - c1(x').  Returns (R, C1, C2), all float64."""
    xt = np.asarray(xt, np.float64)
    d = xt.shape[1]
    if use_opq:
        R, C1 = opq_train(xt, M1, n_outer=n_outer, niter_final=niter, seed=seed)
    else:
        R = np.eye(d)
        C1 = pq_train(xt, M1, niter=niter, seed=seed)
    xr = xt @ R.T
    res = xr - pq_decode(pq_encode(xr, C1, M1), C1, M1)
    C2 = pq_train(res, M2, niter=niter, seed=seed + 500_000)
    return R, C1, C2


def encode(x: np.ndarray, R: np.ndarray, C1: np.ndarray, C2: np.ndarray, M1: int, M2: int):
    """Encode with the two-level codec.  Returns (codes1, codes2, x' = R x, q(x'))."""
    xr = np.asarray(x, np.float64) @ np.asarray(R, np.float64).T
    c1 = pq_encode(xr, C1, M1)
    x1 = pq_decode(c1, C1, M1)
    c2 = pq_encode(xr - x1, C2, M2)
    xh = x1 + pq_decode(c2, C2, M2)
    return c1, c2, xr, xh
