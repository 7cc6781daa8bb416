"""Regression refinement of the oracle: G(x), least-squares weights, the 0-byte shared
weights, the regression codebook trained by EM, and per-vector codeword assignment.
Float64 throughout.

Test infrastructure only (see the package docstring).

Paper passages (Section 4.2, 4.3):
  * G(x) = [q(x), q(g_1(x)), ..., q(g_k(x))], k = 8, the graph neighbours ordered by
    increasing distance to x; the refined vector is beta^T G(x) (rows of G are vectors);
  * 0-byte refinement: one shared beta* minimising sum_x ||x - beta^T G(x)||^2, the
    least-squares solution Y^+ X;
  * regression codebook of B = 256 weight vectors minimising
    L'(B) = sum_x min_beta ||x - beta^T G(x)||^2: k-means on per-vector least-squares
    weights to initialise, then alternate assignment (argmin) and per-cluster least squares.

  * product regression codebook: the coordinates split into M blocks, one codebook per
    block, the block of the estimate being beta^j(x)^T G^j(x) (G^j: the block's columns of
    G); M bytes per vector.  The 0-byte weights beta* per block are the same with one
    codeword per block and nothing stored per vector.

Readings where the paper is silent: a neighbour slot that the graph leaves empty (-1)
contributes a zero row; codeword 0 is reserved as e0 = (1, 0, ..., 0) and never updated,
so that no vector is refined worse than q(x); a small ridge 1e-10 * trace(A) / 9 keeps the
normal equations solvable; an empty cluster keeps its previous codeword; 10 EM iterations
on a seeded subset of at most 250k indexed vectors (Section 5).
"""
from __future__ import annotations

import numpy as np

from .codec import kmeans, splits

KBETA = 8
NBETA = 256


def gmatrix(xh: np.ndarray, adj0: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """G for each index in ``idx``: [n][KBETA+1][d] (row 0 = q(x), rows 1.. = neighbours)."""
    idx = np.asarray(idx, np.int64)
    n, d = idx.shape[0], xh.shape[1]
    G = np.zeros((n, KBETA + 1, d))
    G[:, 0] = xh[idx]
    nb = adj0[idx, :KBETA].astype(np.int64)
    for j in range(min(KBETA, adj0.shape[1])):
        ok = nb[:, j] >= 0
        G[ok, j + 1] = xh[nb[ok, j]]
    return G


def normal_eq(G: np.ndarray, x: np.ndarray):
    """A = G G^T [n][9][9], b = G x [n][9] for the least squares min ||x - beta^T G||^2."""
    A = np.einsum("nid,njd->nij", G, G)
    b = np.einsum("nid,nd->ni", G, x)
    return A, b


def ridge_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    lam = 1e-10 * np.trace(A, axis1=-2, axis2=-1) / A.shape[-1]
    lam = np.where(lam > 0, lam, 1e-300)
    Ar = A + lam[..., None, None] * np.eye(A.shape[-1])
    return np.linalg.solve(Ar, b[..., None])[..., 0]


def beta_star(G: np.ndarray, x: np.ndarray) -> np.ndarray:
    """0-byte refinement weights: one beta for all vectors (least squares over the set)."""
    A, b = normal_eq(G, x)
    return ridge_solve(A.sum(0), b.sum(0))


def losses(G: np.ndarray, x: np.ndarray, B: np.ndarray) -> np.ndarray:
    """||x - beta^T G(x)||^2 for every vector and codeword: [n][len(B)]."""
    Y = np.einsum("bj,njd->nbd", B, G)
    r = x[:, None, :] - Y
    return np.einsum("nbd,nbd->nb", r, r)


def quad_losses(A: np.ndarray, b: np.ndarray, xx: np.ndarray, B: np.ndarray) -> np.ndarray:
    """The same losses from the normal equations: ||x||^2 - 2 beta.b + beta^T A beta."""
    return xx[:, None] - 2.0 * (b @ B.T) + np.einsum("bi,nij,bj->nb", B, A, B, optimize=True)


def assign_codewords(G: np.ndarray, x: np.ndarray, B: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Per-vector codeword index: argmin over the codebook, ties to the lowest index."""
    out = np.empty(x.shape[0], np.int64)
    for a in range(0, x.shape[0], chunk):
        A, b = normal_eq(G[a:a + chunk], x[a:a + chunk])
        xx = (x[a:a + chunk] ** 2).sum(1)
        out[a:a + chunk] = np.argmin(quad_losses(A, b, xx, B), axis=1)
    return out


def e0() -> np.ndarray:
    v = np.zeros(KBETA + 1)
    v[0] = 1.0
    return v


def train_codebook(G: np.ndarray, x: np.ndarray, n_beta: int = NBETA, iters: int = 10,
                   seed: int = 0, history: list | None = None) -> np.ndarray:
    """EM training of the regression codebook on (G, x).  Returns B [n_beta][9]."""
    A, b = normal_eq(G, x)
    per_vec = ridge_solve(A, b)                        # beta(x), least squares per vector
    K = min(n_beta - 1, x.shape[0])
    B = np.tile(e0(), (n_beta, 1))
    if K > 0:
        B[1:1 + K] = kmeans(per_vec, K, niter=25, seed=seed + 31)
    for _ in range(iters):
        a = assign_codewords(G, x, B)                  # assignment step
        if history is not None:
            history.append(float(losses_assigned(G, x, B, a).sum()))
        for i in range(1, n_beta):                     # update step (codeword 0 fixed)
            m = a == i
            if not np.any(m):
                continue
            B[i] = ridge_solve(A[m].sum(0), b[m].sum(0))
        if history is not None:
            history.append(float(losses_assigned(G, x, B, a).sum()))
    return B


def losses_assigned(G: np.ndarray, x: np.ndarray, B: np.ndarray, a: np.ndarray) -> np.ndarray:
    Y = np.einsum("nj,njd->nd", B[a], G)
    r = x - Y
    return np.einsum("nd,nd->n", r, r)


def train_product(G: np.ndarray, x: np.ndarray, n_blocks: int, n_beta: int = NBETA, iters: int = 10,
                  seed: int = 0, history: list | None = None) -> np.ndarray:
    """Product regression codebook (Section 4.3): coordinates split into ``n_blocks``
    contiguous blocks (the PQ split rule: the first d mod M blocks one wider), each block
    with its own codebook of ``n_beta`` weight vectors minimising that block's loss, which is
    the whole loss restricted to the block's coordinates (the losses of the blocks add up).
    ``n_beta`` = 1: the 0-byte weights beta* of Section 4.2, one per block (no per-vector
    code, and no reserved e0).  Returns B [n_blocks][n_beta][9]; ``history`` receives one
    list of EM losses per block."""
    d = x.shape[1]
    off, ln = splits(d, n_blocks)
    B = np.empty((n_blocks, n_beta, KBETA + 1))
    for m in range(n_blocks):
        cols = slice(off[m], off[m] + ln[m])
        Gm, xm = G[:, :, cols], x[:, cols]
        if n_beta == 1:
            B[m, 0] = beta_star(Gm, xm)
        else:
            h: list = []
            B[m] = train_codebook(Gm, xm, n_beta=n_beta, iters=iters, seed=seed + 101 * m, history=h)
            if history is not None:
                history.append(h)
    return B


def assign_product(G: np.ndarray, x: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Per-vector, per-block codeword: argmin of the block's loss, ties to the lowest index.
    Returns [n][n_blocks] (all zero with one codeword per block)."""
    n_blocks, n_beta = B.shape[0], B.shape[1]
    out = np.zeros((x.shape[0], n_blocks), np.int64)
    if n_beta == 1:
        return out
    off, ln = splits(x.shape[1], n_blocks)
    for m in range(n_blocks):
        cols = slice(off[m], off[m] + ln[m])
        out[:, m] = assign_codewords(G[:, :, cols], x[:, cols], B[m])
    return out


def reconstruct(G: np.ndarray, B: np.ndarray, codes: np.ndarray) -> np.ndarray:
    """Refined vectors [n][d]: block m is sum_j B[m][codes[:, m]][j] * G[:, j, block m]."""
    n_blocks = B.shape[0]
    off, ln = splits(G.shape[2], n_blocks)
    out = np.empty((G.shape[0], G.shape[2]))
    for m in range(n_blocks):
        cols = slice(off[m], off[m] + ln[m])
        out[:, cols] = np.einsum("nj,njd->nd", B[m][codes[:, m]], G[:, :, cols])
    return out
